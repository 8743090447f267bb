// LBVH building blocks shared by the per-geometry build (build.cu) and the batched
// persistent build (batch.cu): primitive boxes and centroids, centroid bounds, Morton
// codes, Karras hierarchy emission and the bottom-up fit, each as the work of one
// element so that a kernel or a work item can run it over any range.
//
// Method: Karras, "Maximizing Parallelism in the Construction of BVHs, Octrees, and
// k-d Trees" (HPG 2012); the paper's BVH construction and refit (Sec. 6.2).
#pragma once

#include "grt_internal.cuh"

namespace grt {

// ======================================================================= primitive boxes (A1) and bounds (A2)
struct Box3 {
    float3 lo, hi;
};

__device__ __forceinline__ float3 load3(const char* base, size_t byteOffset) {
    const float* p = reinterpret_cast<const float*>(base + byteOffset);
    return make_float3(p[0], p[1], p[2]);
}

__device__ __forceinline__ Box3 triangleBox(float3 a, float3 b, float3 c) {
    Box3 r;
    r.lo = make_float3(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y), fminf(fminf(a.z, b.z), c.z));
    r.hi = make_float3(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y), fmaxf(fmaxf(a.z, b.z), c.z));
    return r;
}

__device__ __forceinline__ float3 boxCentroid(const Box3& b) {
    return make_float3(__fmul_rn(0.5f, __fadd_rn(b.lo.x, b.hi.x)), __fmul_rn(0.5f, __fadd_rn(b.lo.y, b.hi.y)),
                       __fmul_rn(0.5f, __fadd_rn(b.lo.z, b.hi.z)));
}

struct PrimSource {
    uint32_t kind;  // 0 triangles, 1 boxes at stride, 2 references to split triangles
    uint32_t count; // primitives (kind 2: references)
    const char* idx;
    uint32_t idxStride;
    const char* verts;
    uint32_t vertStride;
    const char* boxes;
    uint32_t boxStride;
    const float4* refs;  // kind 2: two float4 per reference, {lo.xyz, triangle}, {hi.xyz, owner}
};

__device__ __forceinline__ void loadTriangle(const PrimSource& S, uint32_t t, float3* v) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(S.idx + (size_t)t * S.idxStride);
    v[0] = load3(S.verts, (size_t)w[0] * S.vertStride);
    v[1] = load3(S.verts, (size_t)w[1] * S.vertStride);
    v[2] = load3(S.verts, (size_t)w[2] * S.vertStride);
}

// Triangle of reference i (kind 2), and whether i is that triangle's first reference.
__device__ __forceinline__ uint32_t refTriangle(const PrimSource& S, uint32_t i, bool* owner) {
    *owner = __float_as_uint(__ldg(&S.refs[2 * (size_t)i + 1].w)) != 0u;
    return __float_as_uint(__ldg(&S.refs[2 * (size_t)i].w));
}

// Box of primitive (or reference) i; v receives a triangle's vertices (kinds 0 and 2).
__device__ __forceinline__ Box3 primBox(const PrimSource& S, uint32_t i, float3* v) {
    if (S.kind == 0) {
        loadTriangle(S, i, v);
        return triangleBox(v[0], v[1], v[2]);
    }
    if (S.kind == 2) {
        const float4 a = S.refs[2 * (size_t)i], b = S.refs[2 * (size_t)i + 1];
        loadTriangle(S, __float_as_uint(a.w), v);
        Box3 r;
        r.lo = make_float3(a.x, a.y, a.z);
        r.hi = make_float3(b.x, b.y, b.z);
        return r;
    }
    const float* b = reinterpret_cast<const float*>(S.boxes + (size_t)i * S.boxStride);
    Box3 r;
    r.lo = make_float3(b[0], b[1], b[2]);
    r.hi = make_float3(b[3], b[4], b[5]);
    return r;
}

// Block-wide min/max reduction of per-thread bounds folded into 6 ordered-int atomics
// (every thread of the block calls it).
__device__ __forceinline__ void reduceBoxBounds(float mn[3], float mx[3], uint32_t* bounds) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    __shared__ float sm[32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) sm[warp][a] = mn[a], sm[warp][3 + a] = mx[a];
    __syncthreads();
    if (warp == 0) {
        for (int a = 0; a < 3; ++a) {
            mn[a] = lane < nw ? sm[lane][a] : INFINITY;
            mx[a] = lane < nw ? sm[lane][3 + a] : -INFINITY;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
                mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
            }
        if (lane == 0)
            for (int a = 0; a < 3; ++a) {
                atomicMin(&bounds[a], floatToOrdered(mn[a]));
                atomicMax(&bounds[3 + a], floatToOrdered(mx[a]));
            }
    }
}

// Block-wide min/max of centroids (one per thread, `valid` ones only) into the bounds.
__device__ __forceinline__ void reduceBounds(float3 c, bool valid, uint32_t* bounds) {
    float mn[3] = {valid ? c.x : INFINITY, valid ? c.y : INFINITY, valid ? c.z : INFINITY};
    float mx[3] = {valid ? c.x : -INFINITY, valid ? c.y : -INFINITY, valid ? c.z : -INFINITY};
    reduceBoxBounds(mn, mx, bounds);
}

// ======================================================================= Morton codes (A3)
__device__ __forceinline__ uint32_t expand10(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ unsigned long long expand21(uint32_t v) {
    unsigned long long x = v & 0x1FFFFFull;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// q = clamp(floor(((c - lo) / (hi - lo)) * 2^bits), 0, 2^bits - 1), each step rounded
// to nearest in float32; a zero extent gives 0.
template <int BITS>
__device__ __forceinline__ uint32_t quantise(float c, float lo, float hi) {
    const float ext = __fsub_rn(hi, lo);
    const float x = (ext == 0.0f) ? 0.0f : __fdiv_rn(__fsub_rn(c, lo), ext);
    const float s = __fmul_rn(x, (float)(1u << BITS));
    const float f = floorf(s);
    const float top = (float)((1u << BITS) - 1u);
    if (!(f >= 0.0f)) return 0u;
    return (uint32_t)(f > top ? top : f);
}

// Morton code of centroid c inside the centroid bounds (6 ordered-int words: lo xyz, hi xyz).
template <typename K, int BITS>
__device__ __forceinline__ K mortonCode(float4 c, const uint32_t* bounds6) {
    const float lx = orderedToFloat(bounds6[0]), ly = orderedToFloat(bounds6[1]), lz = orderedToFloat(bounds6[2]);
    const float hx = orderedToFloat(bounds6[3]), hy = orderedToFloat(bounds6[4]), hz = orderedToFloat(bounds6[5]);
    const uint32_t qx = quantise<BITS>(c.x, lx, hx), qy = quantise<BITS>(c.y, ly, hy), qz = quantise<BITS>(c.z, lz, hz);
    if constexpr (BITS == 10)
        return (K)((expand10(qx) << 2) | (expand10(qy) << 1) | expand10(qz));
    else
        return (K)((expand21(qx) << 2) | (expand21(qy) << 1) | expand21(qz));
}

// ======================================================================= Karras emission (A5)
// Loads of data written earlier in the same launch by other blocks bypass L1 (CG).
template <bool CG, typename T>
__device__ __forceinline__ T loadData(const T* p) {
    if constexpr (CG) return __ldcg(p);
    return *p;
}

template <bool CG, typename K>
__device__ __forceinline__ int commonPrefix(const K* __restrict__ keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const K a = loadData<CG>(keys + i), b = loadData<CG>(keys + j);
    constexpr int KB = (int)sizeof(K) * 8;
    if (a != b) {
        if (sizeof(K) == 4) return __clz((uint32_t)(a ^ b));
        return __clzll((long long)(a ^ b));
    }
    return KB + __clz((uint32_t)i ^ (uint32_t)j);
}

// One thread per internal node i in [0, n-2]: direction, range end, split; writes
// the node's child indices (word 3 of the node) and each child's parent entry
// (parent << 1 | side).
//
// With sChild / sParent (a single-block build) the child words and parent entries are
// also written to those shared-memory copies.
// Internal node i's child words (leaf bit on leaf children) and its leaf range [first,
// last] (Karras 2012: direction, range end, split).
template <bool CG, typename K>
__device__ __forceinline__ void karrasSplit(const K* __restrict__ keys, int n, int i, uint32_t& left, uint32_t& right,
                                            int& first, int* last = nullptr) {
    const int d = (commonPrefix<CG>(keys, n, i, i + 1) - commonPrefix<CG>(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = commonPrefix<CG>(keys, n, i, i - d);
    int lmax = 2;
    while (commonPrefix<CG>(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (commonPrefix<CG>(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = commonPrefix<CG>(keys, n, i, j);
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (commonPrefix<CG>(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    left = (lo == gamma) ? (kLeafBit | (uint32_t)gamma) : (uint32_t)gamma;
    right = (hi == gamma + 1) ? (kLeafBit | (uint32_t)(gamma + 1)) : (uint32_t)(gamma + 1);
    first = lo;
    if (last) *last = hi;
}

template <bool CG, typename K>
__device__ __forceinline__ void karrasNode(const K* __restrict__ keys, int n, int i, float4* __restrict__ nodes,
                                           uint32_t* __restrict__ parents, uint2* sChild = nullptr,
                                           uint32_t* sParent = nullptr) {
    uint32_t left, right;
    int first;
    karrasSplit<CG>(keys, n, i, left, right, first);
    nodes[4 * (size_t)i + 3] = make_float4(__uint_as_float(left), __uint_as_float(right), 0.f, 0.f);
    const uint32_t leafBase = (uint32_t)n - 1u;
    const uint32_t pl = (left & kLeafBit) ? leafBase + (left & ~kLeafBit) : left;
    const uint32_t pr = (right & kLeafBit) ? leafBase + (right & ~kLeafBit) : right;
    parents[pl] = ((uint32_t)i << 1) | 0u;
    parents[pr] = ((uint32_t)i << 1) | 1u;
    if (i == 0) parents[0] = kInvalid;
    if (sChild) {
        sChild[i] = make_uint2(left, right);
        sParent[pl] = ((uint32_t)i << 1) | 0u;
        sParent[pr] = ((uint32_t)i << 1) | 1u;
        if (i == 0) sParent[0] = kInvalid;
    }
}

// ======================================================================= bottom-up fit (A6) + leaf layout (A7)
struct FitParams {
    PrimSource src;
    uint32_t n;
    const uint32_t* sortedPrims;  // nullptr for a refit (IDs read back from the leaves)
    float4* nodes;
    float4* wide;  // 4-wide nodes, one per binary internal node (kWideWords float4 each)
    void* leaves;
    uint32_t* primToLeaf;
    const uint32_t* parents;
    uint32_t* flags;
    BvhHeader* header;
    const float4* instBoxes;              // scene: world boxes (2 float4 per instance)
    const InstanceRecord* instRecords;    // scene: unsorted records
};

__device__ __forceinline__ void writeChildBox(float4* nodes, uint32_t p, uint32_t side, const Box3& b) {
    float2* n2 = reinterpret_cast<float2*>(nodes + 4 * (size_t)p);
    n2[0 * 2 + side] = make_float2(b.lo.x, b.hi.x);
    n2[1 * 2 + side] = make_float2(b.lo.y, b.hi.y);
    n2[2 * 2 + side] = make_float2(b.lo.z, b.hi.z);
}

// Slots 2t and 2t+1 of 4-wide node w: two boxes (a, b) and their child words (kNone
// with an empty box for an empty slot). Layout of a wide node (kWideWords float4): lo.x
// of slots 0-3, hi.x, lo.y, hi.y, lo.z, hi.z, the four child words, then one unused
// float4; a slot pair is one 8-byte store per row.
__device__ __forceinline__ void writeWidePair(float4* wide, uint32_t w, uint32_t t, float3 alo, float3 ahi, uint32_t ca,
                                              float3 blo, float3 bhi, uint32_t cb) {
    float2* f = reinterpret_cast<float2*>(wide + kWideWords * (size_t)w) + t;
    f[0] = make_float2(alo.x, blo.x);
    f[2] = make_float2(ahi.x, bhi.x);
    f[4] = make_float2(alo.y, blo.y);
    f[6] = make_float2(ahi.y, bhi.y);
    f[8] = make_float2(alo.z, blo.z);
    f[10] = make_float2(ahi.z, bhi.z);
    reinterpret_cast<uint2*>(f)[12] = make_uint2(ca, cb);
}

// ======================================================================= quantised 4-wide nodes (A7)
// Wide node w in 64 bytes (kQuantWords float4): each slot's box as 8-bit planes on a
// per-axis grid of the node's own box (the compressed wide node of Ylitie, Karras and
// Laine, HPG 2017; the paper's wide trees, Sec. 6.2). Per axis, over the used slots:
// origin p = the least slot lo; step 2^e with e the least integer in [-126, 127] for
// which fl(p + 255 2^e) reaches the greatest slot hi; a slot's lower plane is the largest
// q in [0, 255] with fl(p + q 2^e) <= lo, its upper plane the smallest with
// fl(p + q 2^e) >= hi (fl: float32 rounding to nearest; q 2^e is exact, so fl applies
// once). Each condition is monotone, so every choice is unique whatever the starting
// estimate, and the decoded box contains the exact one. Words: p.xyz; the biased
// exponents e + 127 in bytes 0-2; qlo.x, qhi.x, qlo.y, qhi.y, qlo.z, qhi.z (slot j in
// byte j; an empty slot 255 / 0); the four child words; two zero words.
__device__ __forceinline__ float quantDecode(float p, uint32_t q, int e) {
    return __fadd_rn(p, __fmul_rn((float)q, __uint_as_float((uint32_t)(e + 127) << 23)));
}

// Reads wide node W (7 float4, with L1-bypassing loads: it may have been written
// earlier in the same launch) and writes its quantised form to Q.
__device__ __forceinline__ void quantizeWideNode(const float4* W, float4* Q) {
    float4 r[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) r[i] = __ldcg(W + i);
    const uint32_t c[4] = {__float_as_uint(r[6].x), __float_as_uint(r[6].y), __float_as_uint(r[6].z),
                           __float_as_uint(r[6].w)};
    bool used[4];
    bool any = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) any |= (used[j] = c[j] != kInvalid);
    float p3[3];
    uint32_t expWord = 0, planes[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo[4] = {r[2 * a].x, r[2 * a].y, r[2 * a].z, r[2 * a].w};
        const float hi[4] = {r[2 * a + 1].x, r[2 * a + 1].y, r[2 * a + 1].z, r[2 * a + 1].w};
        float p = 0.f, top = 0.f;
        if (any) {
            p = INFINITY, top = -INFINITY;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (used[j]) p = fminf(p, lo[j]), top = fmaxf(top, hi[j]);
        }
        int e = -126;
        if (any) {
            const float ext = __fsub_ru(top, p);
            if (ext > 0.f) {  // a starting estimate: 255 2^e > ext
                const int lg = ilogbf(ext * (1.0f / 255.0f));
                e = lg >= 126 ? 127 : max(-126, lg + 1);
            }
            while (e > -126 && quantDecode(p, 255u, e - 1) >= top) --e;
            while (e < 127 && quantDecode(p, 255u, e) < top) ++e;
        }
        const float inv = __uint_as_float((uint32_t)(127 - e) << 23);  // 2^-e, for the estimates (0 when e = 127)
        uint32_t qlo = 0, qhi = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t ql = 255u, qh = 0u;
            if (used[j]) {
                const float l = lo[j], h = hi[j];
                float g = floorf(__fmul_rn(__fsub_rd(l, p), inv));
                int q = isnan(g) ? 0 : (int)fminf(fmaxf(g, 0.f), 255.f);
                while (q > 0 && quantDecode(p, (uint32_t)q, e) > l) --q;
                while (q < 255 && quantDecode(p, (uint32_t)q + 1u, e) <= l) ++q;
                ql = (uint32_t)q;
                g = ceilf(__fmul_rn(__fsub_ru(h, p), inv));
                q = isnan(g) ? 255 : (int)fminf(fmaxf(g, 0.f), 255.f);
                while (q < 255 && quantDecode(p, (uint32_t)q, e) < h) ++q;
                while (q > 0 && quantDecode(p, (uint32_t)q - 1u, e) >= h) --q;
                qh = (uint32_t)q;
            }
            qlo |= ql << (8 * j);
            qhi |= qh << (8 * j);
        }
        p3[a] = p;
        expWord |= (uint32_t)(e + 127) << (8 * a);
        planes[2 * a] = qlo;
        planes[2 * a + 1] = qhi;
    }
    Q[0] = make_float4(p3[0], p3[1], p3[2], __uint_as_float(expWord));
    Q[1] = make_float4(__uint_as_float(planes[0]), __uint_as_float(planes[1]), __uint_as_float(planes[2]),
                       __uint_as_float(planes[3]));
    Q[2] = make_float4(__uint_as_float(planes[4]), __uint_as_float(planes[5]), __uint_as_float(c[0]),
                       __uint_as_float(c[1]));
    Q[3] = make_float4(__uint_as_float(c[2]), __uint_as_float(c[3]), 0.f, 0.f);
}

// ======================================================================= 8-wide nodes (A7)
// The 8-wide node of binary node k (kWide8Words float4): k's descendants three levels
// down. Slots 4s..4s+3 come from child s: a leaf child fills slot 4s (4s+1..4s+3 empty);
// an internal child's children t fill slots 4s+2t and 4s+2t+1 with their own two
// children, or with themselves (a leaf) and an empty slot. Rows 4a + 2 side + half hold
// axis a's lower (side 0) or upper (side 1) planes of slots 4 half .. 4 half + 3, rows 12
// and 13 the child words (binary format; kInvalid = empty, box +inf / -inf), rows 14-15
// zero. Built from the binary nodes (read with L1-bypassing loads: they may have been
// written earlier in the same launch). n = the primitive count (1: node 0 holds its leaf
// as both children; the 8-wide node holds it once).
__device__ __forceinline__ void binaryChildren(const float4* nodes, uint32_t k, float lo[2][3], float hi[2][3],
                                               uint32_t w[2]) {
    const float4* N = nodes + 4 * (size_t)k;
    const float4 x = __ldcg(N), y = __ldcg(N + 1), z = __ldcg(N + 2), c = __ldcg(N + 3);
    lo[0][0] = x.x, hi[0][0] = x.y, lo[1][0] = x.z, hi[1][0] = x.w;
    lo[0][1] = y.x, hi[0][1] = y.y, lo[1][1] = y.z, hi[1][1] = y.w;
    lo[0][2] = z.x, hi[0][2] = z.y, lo[1][2] = z.z, hi[1][2] = z.w;
    w[0] = __float_as_uint(c.x), w[1] = __float_as_uint(c.y);
}

__device__ __forceinline__ void wide8Node(const float4* nodes, uint32_t n, uint32_t k, float4* out) {
    float S[8][6];  // per slot lo.xyz, hi.xyz
    uint32_t W[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        W[j] = kInvalid;
#pragma unroll
        for (int a = 0; a < 3; ++a) S[j][a] = INFINITY, S[j][3 + a] = -INFINITY;
    }
    auto put = [&](int j, uint32_t w, const float* l, const float* h) {
        W[j] = w;
#pragma unroll
        for (int a = 0; a < 3; ++a) S[j][a] = l[a], S[j][3 + a] = h[a];
    };
    float cl[2][3], ch[2][3];
    uint32_t cw[2];
    binaryChildren(nodes, k, cl, ch, cw);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (s == 1 && n == 1) break;
        if (cw[s] & kLeafBit) {
            put(4 * s, cw[s], cl[s], ch[s]);
            continue;
        }
        float gl[2][3], gh[2][3];
        uint32_t gw[2];
        binaryChildren(nodes, cw[s], gl, gh, gw);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (gw[t] & kLeafBit) {
                put(4 * s + 2 * t, gw[t], gl[t], gh[t]);
                continue;
            }
            float hl[2][3], hh[2][3];
            uint32_t hw[2];
            binaryChildren(nodes, gw[t], hl, hh, hw);
            put(4 * s + 2 * t, hw[0], hl[0], hh[0]);
            put(4 * s + 2 * t + 1, hw[1], hl[1], hh[1]);
        }
    }
    float4* O = out + kWide8Words * (size_t)k;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int side = 0; side < 2; ++side)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = 3 * side + a;
                O[4 * a + 2 * side + h] = make_float4(S[4 * h][q], S[4 * h + 1][q], S[4 * h + 2][q], S[4 * h + 3][q]);
            }
    O[12] = make_float4(__uint_as_float(W[0]), __uint_as_float(W[1]), __uint_as_float(W[2]), __uint_as_float(W[3]));
    O[13] = make_float4(__uint_as_float(W[4]), __uint_as_float(W[5]), __uint_as_float(W[6]), __uint_as_float(W[7]));
    O[14] = O[15] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Leaf k of the sorted order: writes the leaf record and walks up while this thread is
// the second to reach a node, writing each box into its parent.
//
// The same walk writes the 4-wide nodes. Wide node w has the children of binary node w,
// each internal child replaced by its own two children: slots 2s and 2s+1 hold child
// s's two children, or child s itself (a leaf) and an empty slot. The thread that
// completes binary node p (the second to arrive) reads its two child boxes and writes
// them as slots 2s'+0/1 of wide node g, p's parent (p being g's child s'), and each
// leaf child s of p as slot pair 2s of wide node p. These stores come after the atomic,
// so its release orders only the binary box the sibling's thread reads. Traversal starts
// at wide node 0 and only reaches the wide nodes of binary nodes at even depth; the
// others are written all the same.
//
// BLOCK: every leaf of the build is walked by a thread of one block (the single-block
// build). The visit counters are then `blockFlags` in shared memory and the box
// hand-off is ordered at block scope (fence, shared atomic, fence), so a walk's steps
// stay in the SM instead of making a round trip to L2 per level.
template <int KIND, bool BLOCK = false>  // KIND: 0 triangles, 1 AABB list, 2 instances
__device__ __forceinline__ void fitLeaf(const FitParams& P, uint32_t k, uint32_t* blockFlags = nullptr) {
    Box3 b;
    if (KIND == 0) {
        float4* rec = reinterpret_cast<float4*>(P.leaves) + 3 * (size_t)k;
        const uint32_t item = P.sortedPrims ? __ldcg(P.sortedPrims + k) : __float_as_uint(rec[0].w);
        float3 v[3];
        b = primBox(P.src, item, v);
        bool owner = true;
        const uint32_t prim = P.src.kind == 2 ? refTriangle(P.src, item, &owner) : item;
        rec[0] = make_float4(v[0].x, v[0].y, v[0].z, __uint_as_float(prim));
        // w slots: L1 norms of the edges v1-v0 and v2-v0 (scale of the traversal's error bounds)
        const float e1 = fabsf(v[1].x - v[0].x) + fabsf(v[1].y - v[0].y) + fabsf(v[1].z - v[0].z);
        const float e2 = fabsf(v[2].x - v[0].x) + fabsf(v[2].y - v[0].y) + fabsf(v[2].z - v[0].z);
        rec[1] = make_float4(v[1].x, v[1].y, v[1].z, e1);
        rec[2] = make_float4(v[2].x, v[2].y, v[2].z, e2);
        if (owner) P.primToLeaf[prim] = k;
    } else if (KIND == 1) {
        uint32_t* ids = reinterpret_cast<uint32_t*>(P.leaves);
        const uint32_t prim = P.sortedPrims ? __ldcg(P.sortedPrims + k) : ids[k];
        float3 v[3];
        b = primBox(P.src, prim, v);
        ids[k] = prim;
    } else {
        const uint32_t prim = P.sortedPrims[k];
        const float4 lo = P.instBoxes[2 * (size_t)prim], hi = P.instBoxes[2 * (size_t)prim + 1];
        b.lo = make_float3(lo.x, lo.y, lo.z);
        b.hi = make_float3(hi.x, hi.y, hi.z);
        reinterpret_cast<InstanceRecord*>(P.leaves)[k] = P.instRecords[prim];
        P.primToLeaf[prim] = k;
    }
    if (P.n == 1) {
        // a single primitive: node 0 holds it as both children
        writeChildBox(P.nodes, 0, 0, b);
        writeChildBox(P.nodes, 0, 1, b);
        P.nodes[3] = make_float4(__uint_as_float(kLeafBit), __uint_as_float(kLeafBit), 0.f, 0.f);
        const float3 elo = make_float3(INFINITY, INFINITY, INFINITY), ehi = make_float3(-INFINITY, -INFINITY, -INFINITY);
        writeWidePair(P.wide, 0, 0, b.lo, b.hi, kLeafBit, elo, ehi, kInvalid);
        writeWidePair(P.wide, 0, 1, elo, ehi, kInvalid, elo, ehi, kInvalid);
        P.header->rootLo[0] = b.lo.x, P.header->rootLo[1] = b.lo.y, P.header->rootLo[2] = b.lo.z;
        P.header->rootHi[0] = b.hi.x, P.header->rootHi[1] = b.hi.y, P.header->rootHi[2] = b.hi.z;
        return;
    }
    uint32_t pe = BLOCK ? P.parents[P.n - 1 + k] : __ldcg(P.parents + P.n - 1 + k);
    for (;;) {
        const uint32_t p = pe >> 1, side = pe & 1u;
        writeChildBox(P.nodes, p, side, b);
        uint32_t prev;
        float4 bx, by, bz, bc;
        uint32_t ge;
        if (BLOCK) {
            // message passing at block scope: box store, fence, counter; counter, fence, loads
            __threadfence_block();
            prev = atomicAdd(blockFlags + p, 1u);
            if (prev == 0) return;
            __threadfence_block();
            bx = P.nodes[4 * (size_t)p + 0];
            by = P.nodes[4 * (size_t)p + 1];
            bz = P.nodes[4 * (size_t)p + 2];
            bc = P.nodes[4 * (size_t)p + 3];
            ge = p == 0 ? kInvalid : P.parents[p];
        } else {
            // acquire-release at GPU scope: releases this box to the sibling's thread if it
            // comes second, and acquires the sibling's box if this thread comes second
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(P.flags + p) : "memory");
            if (prev == 0) return;  // the sibling is still on its way up
            bx = __ldcg(&P.nodes[4 * (size_t)p + 0]);
            by = __ldcg(&P.nodes[4 * (size_t)p + 1]);
            bz = __ldcg(&P.nodes[4 * (size_t)p + 2]);
            bc = __ldcg(&P.nodes[4 * (size_t)p + 3]);
            ge = p == 0 ? kInvalid : __ldcg(&P.parents[p]);
        }
        const uint32_t c0 = __float_as_uint(bc.x), c1 = __float_as_uint(bc.y);
        const float3 lo0 = make_float3(bx.x, by.x, bz.x), hi0 = make_float3(bx.y, by.y, bz.y);
        const float3 lo1 = make_float3(bx.z, by.z, bz.z), hi1 = make_float3(bx.w, by.w, bz.w);
        const float3 elo = make_float3(INFINITY, INFINITY, INFINITY), ehi = make_float3(-INFINITY, -INFINITY, -INFINITY);
        if (c0 & kLeafBit) writeWidePair(P.wide, p, 0, lo0, hi0, c0, elo, ehi, kInvalid);
        if (c1 & kLeafBit) writeWidePair(P.wide, p, 1, lo1, hi1, c1, elo, ehi, kInvalid);
        if (ge != kInvalid) writeWidePair(P.wide, ge >> 1, ge & 1u, lo0, hi0, c0, lo1, hi1, c1);
        b.lo = make_float3(fminf(bx.x, bx.z), fminf(by.x, by.z), fminf(bz.x, bz.z));
        b.hi = make_float3(fmaxf(bx.y, bx.w), fmaxf(by.y, by.w), fmaxf(bz.y, bz.w));
        if (p == 0) {
            P.header->rootLo[0] = b.lo.x, P.header->rootLo[1] = b.lo.y, P.header->rootLo[2] = b.lo.z;
            P.header->rootHi[0] = b.hi.x, P.header->rootHi[1] = b.hi.y, P.header->rootHi[2] = b.hi.z;
            return;
        }
        pe = ge;
    }
}

// The fit of a single-block build with every box kept in shared memory, in two steps.
// Node j of the build (internal nodes 0..n-2, then leaf k as n-1+k) has its box in sBox
// (six float arrays of 2n-1 entries: lo.x, lo.y, lo.z, hi.x, hi.y, hi.z), its parent
// entry in sParent and, for internal nodes, its child words in sChild and a visit
// counter in sFlag (zeroed).
//  1. fitLeafShared: leaf k's thread stores its box and walks up while it is the second
//     to reach a node, storing the union for the level above. Only shared memory is
//     touched during the walk (hand-offs ordered at block scope: fence, shared atomic,
//     fence), so no fence waits on a global store; the leaf record is written after.
//  2. writeNodeShared, one thread per internal node after a block barrier: binary node
//     p (child boxes and child words, as emission and the fit write them) and 4-wide
//     node p (p's children, each internal child replaced by its two children).
struct SharedFit {
    float* sBox;  // 6 x (2n-1)
    uint32_t* sParent;
    const uint2* sChild;
    uint32_t* sFlag;
};

__device__ __forceinline__ void storeBoxShared(const SharedFit& F, uint32_t total, uint32_t j, const Box3& b) {
    F.sBox[0 * total + j] = b.lo.x, F.sBox[1 * total + j] = b.lo.y, F.sBox[2 * total + j] = b.lo.z;
    F.sBox[3 * total + j] = b.hi.x, F.sBox[4 * total + j] = b.hi.y, F.sBox[5 * total + j] = b.hi.z;
}

__device__ __forceinline__ Box3 loadBoxShared(const SharedFit& F, uint32_t total, uint32_t j) {
    Box3 b;
    b.lo = make_float3(F.sBox[j], F.sBox[total + j], F.sBox[2 * total + j]);
    b.hi = make_float3(F.sBox[3 * total + j], F.sBox[4 * total + j], F.sBox[5 * total + j]);
    return b;
}

// Node index (0..2n-2) of child word c.
__device__ __forceinline__ uint32_t nodeOfChild(uint32_t c, uint32_t n) {
    return (c & kLeafBit) ? n - 1 + (c & ~kLeafBit) : c;
}

template <int KIND>
__device__ __forceinline__ void fitLeafShared(const FitParams& P, uint32_t k, const SharedFit& F) {
    const uint32_t n = P.n, total = 2 * n - 1;
    Box3 b;
    uint32_t prim = P.sortedPrims[k];
    float3 v[3];
    if (KIND == 2) {
        const float4 lo = P.instBoxes[2 * (size_t)prim], hi = P.instBoxes[2 * (size_t)prim + 1];
        b.lo = make_float3(lo.x, lo.y, lo.z);
        b.hi = make_float3(hi.x, hi.y, hi.z);
    } else {
        b = primBox(P.src, prim, v);
    }
    uint32_t j = n - 1 + k;
    for (;;) {
        storeBoxShared(F, total, j, b);
        if (j == 0) {
            P.header->rootLo[0] = b.lo.x, P.header->rootLo[1] = b.lo.y, P.header->rootLo[2] = b.lo.z;
            P.header->rootHi[0] = b.hi.x, P.header->rootHi[1] = b.hi.y, P.header->rootHi[2] = b.hi.z;
            break;
        }
        const uint32_t p = F.sParent[j] >> 1;
        __threadfence_block();
        if (atomicAdd(F.sFlag + p, 1u) == 0) break;  // the sibling is still on its way up
        __threadfence_block();
        const uint2 c = F.sChild[p];
        const Box3 b0 = loadBoxShared(F, total, nodeOfChild(c.x, n)), b1 = loadBoxShared(F, total, nodeOfChild(c.y, n));
        b.lo = make_float3(fminf(b0.lo.x, b1.lo.x), fminf(b0.lo.y, b1.lo.y), fminf(b0.lo.z, b1.lo.z));
        b.hi = make_float3(fmaxf(b0.hi.x, b1.hi.x), fmaxf(b0.hi.y, b1.hi.y), fmaxf(b0.hi.z, b1.hi.z));
        j = p;
    }
    if (KIND == 0) {
        float4* rec = reinterpret_cast<float4*>(P.leaves) + 3 * (size_t)k;
        rec[0] = make_float4(v[0].x, v[0].y, v[0].z, __uint_as_float(prim));
        // w slots: L1 norms of the edges v1-v0 and v2-v0 (scale of the traversal's error bounds)
        const float e1 = fabsf(v[1].x - v[0].x) + fabsf(v[1].y - v[0].y) + fabsf(v[1].z - v[0].z);
        const float e2 = fabsf(v[2].x - v[0].x) + fabsf(v[2].y - v[0].y) + fabsf(v[2].z - v[0].z);
        rec[1] = make_float4(v[1].x, v[1].y, v[1].z, e1);
        rec[2] = make_float4(v[2].x, v[2].y, v[2].z, e2);
        P.primToLeaf[prim] = k;
    } else if (KIND == 1) {
        reinterpret_cast<uint32_t*>(P.leaves)[k] = prim;
    } else {
        reinterpret_cast<InstanceRecord*>(P.leaves)[k] = P.instRecords[prim];
        P.primToLeaf[prim] = k;
    }
}

// Component `comp` (0..5: lo.x, hi.x, lo.y, hi.y, lo.z, hi.z) of node j's box.
__device__ __forceinline__ float boxComp(const SharedFit& F, uint32_t total, uint32_t j, uint32_t comp) {
    return F.sBox[((comp & 1u) ? 3u : 0u) * total + (comp >> 1) * total + j];
}

// Row r of binary node p (0..2: the x, y, z rows (c0.lo, c0.hi, c1.lo, c1.hi); 3: the
// child words and two zero words), from the shared boxes and child words.
__device__ __forceinline__ float4 binaryRowShared(const SharedFit& F, uint32_t n, uint32_t p, uint32_t r) {
    const uint32_t total = 2 * n - 1;
    const uint2 c = F.sChild[p];
    if (r == 3) return make_float4(__uint_as_float(c.x), __uint_as_float(c.y), 0.f, 0.f);
    const uint32_t j0 = nodeOfChild(c.x, n), j1 = nodeOfChild(c.y, n);
    return make_float4(boxComp(F, total, j0, 2 * r), boxComp(F, total, j0, 2 * r + 1), boxComp(F, total, j1, 2 * r),
                       boxComp(F, total, j1, 2 * r + 1));
}

// Row r of 4-wide node p (0..5: component r of the four slots; 6: the four child words;
// 7: zero): slots 2s and 2s+1 hold child s's two children, or child s itself (a leaf)
// and an empty slot (child word kInvalid, box +inf / -inf).
__device__ __forceinline__ float4 wideRowShared(const SharedFit& F, uint32_t n, uint32_t p, uint32_t r) {
    const uint32_t total = 2 * n - 1;
    if (r == 7) return make_float4(0.f, 0.f, 0.f, 0.f);
    const uint2 c = F.sChild[p];
    const uint32_t cw[2] = {c.x, c.y};
    float out[4];
#pragma unroll
    for (uint32_t s = 0; s < 2; ++s) {
        uint32_t a, b;
        if (cw[s] & kLeafBit) {
            a = cw[s], b = kInvalid;
        } else {
            const uint2 g = F.sChild[cw[s]];
            a = g.x, b = g.y;
        }
        if (r == 6) {
            out[2 * s] = __uint_as_float(a), out[2 * s + 1] = __uint_as_float(b);
        } else {
            out[2 * s] = boxComp(F, total, nodeOfChild(a, n), r);
            out[2 * s + 1] = b == kInvalid ? ((r & 1u) ? -INFINITY : INFINITY) : boxComp(F, total, nodeOfChild(b, n), r);
        }
    }
    return make_float4(out[0], out[1], out[2], out[3]);
}

// Host: checks a geometry build input and returns its primitive count; the device-side
// description of its primitives.
grtError validateGeometryInput(const grtGeometryBuildInput* in, uint32_t* count);
PrimSource primSource(const grtGeometryBuildInput* in, uint32_t count);

}  // namespace grt
