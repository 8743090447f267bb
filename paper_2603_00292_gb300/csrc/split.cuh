// Spatial splits of triangles before a build (GRT_BUILD_SPLIT_TRIANGLES): the paper's
// high-quality option names spatial splits (Sec. 8, SBVH); they are made here ahead of
// the build, after Karras and Aila ("Fast Parallel Construction of High-Quality Bounding
// Volume Hierarchies", HPG 2013): a budget S of extra references is shared out by a
// per-triangle priority, and each triangle is cut recursively at the most important
// plane of a 1024-cell grid over the scene that crosses its box. The build then runs
// over the n + S references (PrimSource kind 2) exactly as over primitives.
//
// Seven steps (launches of build.cu's per-geometry kernels, or phases of the batched
// launch), one thread per triangle where not said: the scene box; the weights
// (integer cube roots of the priority) and their per-chunk sums; one block's exclusive
// scan of those sums (and the total W); each triangle's share of the budget from its
// place in the running sum of weights, floor(S C_{t+1} / W) - floor(S C_t / W), and
// per-chunk sums of the shares; one block's scan of those; each triangle's first slot
// and the triangle of every slot; then one thread per reference, which walks down its
// triangle's cut tree to its leaf and writes the reference, its centroid and the
// centroid bounds. A thread per reference keeps the lanes of a warp busy however
// unevenly the splits fall (a thread per triangle would wait on the most-split one).
// The arithmetic is float32 (GB300's FP64 rate is a small fraction of its FP32 rate),
// every operation an explicit round-to-nearest intrinsic (nothing is fused), min / max
// written as selections and the integer steps exact, so the results are bit-for-bit
// those of any sequential IEEE-754 evaluation of the same steps.
#pragma once

#include "lbvh.cuh"

namespace grt {

constexpr int kSplitMax = 31;               // splits one triangle takes by priority (+1 from the remainder)
constexpr int kSplitThreads = 256;
constexpr int kSplitScanThreads = 1024;

struct SplitParams {
    PrimSource src;                // the triangles (idx / verts)
    uint32_t n;                    // triangles
    uint32_t budget;               // S
    uint32_t* sceneBounds;         // 6 ordered words: union of the triangle boxes
    unsigned long long* totals;    // [0] sum of the weights W, [1] splits handed out by priority, [2] 1 / W (double)
    uint32_t* counts;              // per triangle: its weight, then its priority splits
    unsigned long long* weightSums;  // per block of kSplitThreads triangles: weights, then their exclusive prefix
    uint32_t* blockSums;           // per block: splits, then their exclusive prefix
    uint32_t blocks;
    float4* refs;                  // (n + S) x {lo.xyz, triangle}, {hi.xyz, owner}
    float4* centroids;             // (n + S)
    uint32_t* centroidBounds;      // 6 ordered words
    uint32_t* firstSlot;           // per triangle: its first reference
    uint32_t* slotTriangle;        // per reference: its triangle
    uint32_t* error;               // device error word
};

struct SBox {
    float lo[3], hi[3];
};

__device__ __forceinline__ float selMin(float a, float b) { return b < a ? b : a; }
__device__ __forceinline__ float selMax(float a, float b) { return a < b ? b : a; }

struct SplitGrid {
    float lo[3], ext[3], inv[3];
    float ghi[3];
};

__device__ __forceinline__ SplitGrid loadSplitGrid(const uint32_t* b6) {
    SplitGrid g;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = orderedToFloat(__ldcg(b6 + a));
        g.ghi[a] = orderedToFloat(__ldcg(b6 + 3 + a));
        g.ext[a] = __fsub_rn(g.ghi[a], g.lo[a]);
        g.inv[a] = g.ext[a] > 0.0f ? __fdiv_rn(1024.0f, g.ext[a]) : 0.0f;
    }
    return g;
}

// Cell of coordinate x on axis a: floor(q), or ceil(q) - 1 for the end of a box
// (a box ending on a grid line does not reach the next cell), clamped to [0, 1023].
__device__ __forceinline__ int gridCell(const SplitGrid& g, float x, int a, bool end) {
    if (g.inv[a] == 0.0f) return 0;
    const float q = __fmul_rn(__fsub_rn(x, g.lo[a]), g.inv[a]);
    const float f = end ? __fsub_rn(ceilf(q), 1.0f) : floorf(q);
    if (!(f >= 0.0f)) return 0;
    if (f > 1023.0f) return 1023;
    return (int)f;
}

// First and last cell of box b on axis a, the box narrowed at each end by 2^-18 of its
// coordinates' magnitude (more than the widening of a crossing).
__device__ __forceinline__ void gridSpan(const SplitGrid& g, const SBox& b, int a, int* cl, int* ch) {
    const float d = __fmul_rn(selMax(fabsf(b.lo[a]), fabsf(b.hi[a])), 0x1p-18f);
    *cl = gridCell(g, __fadd_rn(b.lo[a], d), a, false);
    const int e = gridCell(g, __fsub_rn(b.hi[a], d), a, true);
    *ch = e > *cl ? e : *cl;
}

__device__ __forceinline__ int bitLength(uint32_t x) { return 32 - __clz(x); }

// Largest w with w^3 <= N (N <= 2^63): a float estimate (within one of the root), then
// exact integer steps.
__device__ __forceinline__ uint32_t integerCubeRoot(unsigned long long N) {
    unsigned long long w = (unsigned long long)cbrtf((float)N);
    for (int i = 0; i < 4 && w > 0 && w * w * w > N; ++i) --w;
    for (int i = 0; i < 4 && (w + 1) * (w + 1) * (w + 1) <= N; ++i) ++w;
    return (uint32_t)w;
}

// floor(S X / W) exactly, for 0 < W < 2^63 and X <= W, given invW ~ 1 / W: a double
// estimate (off by at most one) corrected against the 128-bit product S X.
__device__ __forceinline__ unsigned long long mulDivFloor(uint32_t S, unsigned long long X, unsigned long long W,
                                                          double invW) {
    const unsigned long long ph = __umul64hi((unsigned long long)S, X), pl = (unsigned long long)S * X;
    unsigned long long q = (unsigned long long)__dmul_rn(__dmul_rn((double)S, (double)X), invW);
    for (int i = 0; i < 4; ++i) {  // q W <= S X
        const unsigned long long h = __umul64hi(q, W), l = q * W;
        if (q > 0 && (h > ph || (h == ph && l > pl)))
            --q;
        else
            break;
    }
    for (int i = 0; i < 4; ++i) {  // (q + 1) W > S X
        const unsigned long long h = __umul64hi(q + 1, W), l = (q + 1) * W;
        if (h < ph || (h == ph && l <= pl))
            ++q;
        else
            break;
    }
    return q;
}

__device__ __forceinline__ float halfArea(const SBox& b) {
    const float dx = __fsub_rn(b.hi[0], b.lo[0]), dy = __fsub_rn(b.hi[1], b.lo[1]), dz = __fsub_rn(b.hi[2], b.lo[2]);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
}

__device__ __forceinline__ float longestExtent(const SBox& b) {
    float w = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) w = selMax(w, __fsub_rn(b.hi[a], b.lo[a]));
    return w;
}

__device__ __forceinline__ bool boxEmpty(const SBox& b) {
    return b.lo[0] > b.hi[0] || b.lo[1] > b.hi[1] || b.lo[2] > b.hi[2];
}

__device__ __forceinline__ void splitTriangle(const PrimSource& S, uint32_t t, float v[3][3], SBox* box) {
    float3 w[3];
    loadTriangle(S, t, w);
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i][0] = w[i].x, v[i][1] = w[i].y, v[i][2] = w[i].z;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        box->lo[a] = selMin(selMin(v[0][a], v[1][a]), v[2][a]);
        box->hi[a] = selMax(selMax(v[0][a], v[1][a]), v[2][a]);
    }
}

// The cutting plane of box b: the grid line of the highest level inside it (ties:
// longer extent, then lower axis), else the midpoint of its longest axis.
__device__ __forceinline__ void cutPlane(const SplitGrid& g, const SBox& b, int* axis, float* plane) {
    int best = -1, bestBit = -1, bestJ = 0;
    float bestExt = -1.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int cl, ch;
        gridSpan(g, b, a, &cl, &ch);
        if (cl == ch) continue;
        const int bit = bitLength((uint32_t)(cl ^ ch)) - 1;
        const float e = __fsub_rn(b.hi[a], b.lo[a]);
        if (bit > bestBit || (bit == bestBit && e > bestExt)) best = a, bestBit = bit, bestExt = e, bestJ = (ch >> bit) << bit;
    }
    if (best >= 0) {
        *axis = best;
        *plane = __fadd_rn(g.lo[best], __fmul_rn((float)bestJ, __fmul_rn(g.ext[best], 0x1p-10f)));
        return;
    }
    int a0 = 0;
    float e0 = __fsub_rn(b.hi[0], b.lo[0]);
#pragma unroll
    for (int a = 1; a < 3; ++a) {
        const float e = __fsub_rn(b.hi[a], b.lo[a]);
        if (e > e0) a0 = a, e0 = e;
    }
    *axis = a0;
    *plane = __fmul_rn(0.5f, __fadd_rn(b.lo[a0], b.hi[a0]));
}

// Boxes of the triangle's parts on the two sides of x_axis = P, each within b: the
// vertices on that side (<= / >=), then the edge crossings, computed once for both sides
// and widened by pad = 2^-19 of the endpoints' magnitude (+ 2^-140): the float rounding
// of a crossing stays below 12 units in the last place of that magnitude, so the
// widened interval holds the exact crossing.
__device__ __forceinline__ void clipBoth(const float v[3][3], int axis, float P, const SBox& b, SBox* L, SBox* R) {
#pragma unroll
    for (int c = 0; c < 3; ++c) L->lo[c] = R->lo[c] = INFINITY, L->hi[c] = R->hi[c] = -INFINITY;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool l = v[i][axis] <= P, r = v[i][axis] >= P;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (l) L->lo[c] = selMin(L->lo[c], v[i][c]), L->hi[c] = selMax(L->hi[c], v[i][c]);
            if (r) R->lo[c] = selMin(R->lo[c], v[i][c]), R->hi[c] = selMax(R->hi[c], v[i][c]);
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float* a = v[i];
        const float* e = v[i == 2 ? 0 : i + 1];
        const bool crosses = (a[axis] < P && e[axis] > P) || (a[axis] > P && e[axis] < P);
        if (!crosses) continue;
        const float t = __fdiv_rn(__fsub_rn(P, a[axis]), __fsub_rn(e[axis], a[axis]));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float lo = P, hi = P;
            if (c != axis) {
                const float q = __fadd_rn(a[c], __fmul_rn(__fsub_rn(e[c], a[c]), t));
                const float pad = __fadd_rn(__fmul_rn(selMax(fabsf(a[c]), fabsf(e[c])), 0x1p-19f), 0x1p-140f);
                lo = __fsub_rn(q, pad);
                hi = __fadd_rn(q, pad);
            }
            L->lo[c] = selMin(L->lo[c], lo), L->hi[c] = selMax(L->hi[c], hi);
            R->lo[c] = selMin(R->lo[c], lo), R->hi[c] = selMax(R->hi[c], hi);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        L->lo[c] = selMax(L->lo[c], b.lo[c]), L->hi[c] = selMin(L->hi[c], b.hi[c]);
        R->lo[c] = selMax(R->lo[c], b.lo[c]), R->hi[c] = selMin(R->hi[c], b.hi[c]);
    }
}

// One cut of box `cur` (s >= 1 splits left): the two sides' boxes and the left side's
// share sL of the s - 1 splits that remain.
__device__ __forceinline__ void cutOnce(const SplitGrid& g, const float v[3][3], const SBox& cur, int s, SBox* L,
                                        SBox* R, int* sL) {
    int axis;
    float plane;
    cutPlane(g, cur, &axis, &plane);
    clipBoth(v, axis, plane, cur, L, R);
    const int rest = s - 1;
    const bool eL = boxEmpty(*L), eR = boxEmpty(*R);
    if (eL && eR) {
        *L = *R = cur;
        *sL = 0;
    } else if (eL) {
        *L = *R;
        *sL = 0;
    } else if (eR) {
        *R = *L;
        *sL = rest;
    } else {
        const float wL = longestExtent(*L), wR = longestExtent(*R);
        const float sum = __fadd_rn(wL, wR);
        int k = sum > 0.0f ? (int)floorf(__fadd_rn(__fdiv_rn(__fmul_rn((float)rest, wL), sum), 0.5f)) : rest / 2;
        *sL = k < rest ? k : rest;
    }
}

// ----------------------------------------------------------------------- chunk ranges
// Each step is written over a chunk of triangles (or of references) and run by a whole
// block of any size (a multiple of 32), so that the per-geometry kernels below (a chunk
// of 256 triangles per block) and the batched launch's work items (larger chunks) run
// the same code. Sums and scans are exact integers: the chunking changes no result.
// Data an earlier step wrote (in the batched launch: another block of the same launch)
// is read with L1-bypassing loads.

// Exclusive prefix of x over the block and the block's total (every thread calls it;
// its shared words may be reused after a __syncthreads).
template <typename T>
__device__ __forceinline__ T blockExclusive(T x, T* total) {
    __shared__ T warpSums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warpSums[warp] = inc;
    __syncthreads();
    T before = inc - x, all = 0;
    for (int w = 0; w < warps; ++w) {
        if (w < warp) before += warpSums[w];
        all += warpSums[w];
    }
    *total = all;
    return before;
}

// Scene box over triangles [b0, b1).
__device__ __forceinline__ void splitBoundsRange(const SplitParams& P, uint32_t b0, uint32_t b1) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t t = b0 + threadIdx.x; t < b1; t += blockDim.x) {
        float v[3][3];
        SBox b;
        splitTriangle(P.src, t, v, &b);
        for (int a = 0; a < 3; ++a) mn[a] = selMin(mn[a], b.lo[a]), mx[a] = selMax(mx[a], b.hi[a]);
    }
    reduceBoxBounds(mn, mx, P.sceneBounds);
}

// The weight of triangle t (the integer cube root of its priority, 2^53 scaled).
__device__ __forceinline__ uint32_t splitWeight(const SplitParams& P, const SplitGrid& g, uint32_t t) {
    float v[3][3];
    SBox b;
    splitTriangle(P.src, t, v, &b);
    int level = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int cl, ch;
        gridSpan(g, b, a, &cl, &ch);
        const int L = bitLength((uint32_t)(cl ^ ch));
        level = L > level ? L : level;
    }
    float e1[3], e2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) e1[a] = __fsub_rn(v[1][a], v[0][a]), e2[a] = __fsub_rn(v[2][a], v[0][a]);
    const float cx = __fsub_rn(__fmul_rn(e1[1], e2[2]), __fmul_rn(e1[2], e2[1]));
    const float cy = __fsub_rn(__fmul_rn(e1[2], e2[0]), __fmul_rn(e1[0], e2[2]));
    const float cz = __fsub_rn(__fmul_rn(e1[0], e2[1]), __fmul_rn(e1[1], e2[0]));
    const float tri = __fmul_rn(0.5f, __fadd_rn(__fadd_rn(fabsf(cx), fabsf(cy)), fabsf(cz)));
    float excess = __fsub_rn(halfArea(b), tri);
    if (!(excess > 0.0f)) excess = 0.0f;
    SBox G;
    for (int a = 0; a < 3; ++a) G.lo[a] = g.lo[a], G.hi[a] = g.ghi[a];
    const float areaG = halfArea(G);
    const float r = areaG > 0.0f ? __fmul_rn(__fdiv_rn(excess, areaG), (float)(1u << level)) : 0.0f;
    return integerCubeRoot((unsigned long long)__fmul_rn(r, 0x1p53f));  // r 2^53 <= 2^63
}

// Weights of triangles [b0, b1) and their sum, weightSums[chunk].
__device__ __forceinline__ void splitWeightRange(const SplitParams& P, uint32_t chunk, uint32_t b0, uint32_t b1) {
    const SplitGrid g = loadSplitGrid(P.sceneBounds);
    unsigned long long sum = 0;
    for (uint32_t base = b0; base < b1; base += blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        uint32_t w = 0;
        if (t < b1) {
            w = splitWeight(P, g, t);
            P.counts[t] = w;
        }
        unsigned long long roundTotal;
        blockExclusive<unsigned long long>(w, &roundTotal);
        __syncthreads();
        sum += roundTotal;
    }
    if (threadIdx.x == 0) P.weightSums[chunk] = sum;
}

// One block: exclusive prefix sums of `count` per-chunk values, in place; the total
// goes to *total.
template <typename T>
__device__ __forceinline__ void scanBlockSums(T* v, uint32_t count, unsigned long long* total) {
    __shared__ T warpSums[32];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    for (uint32_t base = 0; base < count; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const T x = i < count ? __ldcg(v + i) : (T)0;
        T inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warpSums[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            T ws = lane < warps ? warpSums[lane] : (T)0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T y = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += y;
            }
            if (lane < warps) warpSums[lane] = ws;  // inclusive over warps
        }
        __syncthreads();
        const T before = carry + (warp ? warpSums[warp - 1] : (T)0) + inc - x;
        if (i < count) v[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += warpSums[warps - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = (unsigned long long)carry;
}

// The weight scan over `chunks` chunks, W and 1 / W.
__device__ __forceinline__ void splitScanWeights(const SplitParams& P, uint32_t chunks) {
    scanBlockSums<unsigned long long>(P.weightSums, chunks, P.totals);
    __syncthreads();
    if (threadIdx.x == 0 && P.totals[0])  // 1 / W for the estimates of the shares
        reinterpret_cast<double*>(P.totals)[2] = __ddiv_rn(1.0, (double)P.totals[0]);
}

// Splits by priority of triangles [b0, b1): each one's share of the budget between the
// running weight sums before and after it, capped at kSplitMax; their sum blockSums[chunk].
__device__ __forceinline__ void splitCountRange(const SplitParams& P, uint32_t chunk, uint32_t b0, uint32_t b1) {
    const unsigned long long W = __ldcg(P.totals);
    const double invW = W ? __ldcg(reinterpret_cast<const double*>(P.totals) + 2) : 0.0;
    unsigned long long carry = __ldcg(P.weightSums + chunk);
    uint32_t sum = 0;
    for (uint32_t base = b0; base < b1; base += blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        const unsigned long long w = t < b1 ? __ldcg(P.counts + t) : 0ull;
        unsigned long long roundTotal;
        const unsigned long long local = blockExclusive<unsigned long long>(w, &roundTotal);
        uint32_t s = 0;
        if (t < b1) {
            if (W) {
                const unsigned long long C = carry + local;
                const unsigned long long q = mulDivFloor(P.budget, C + w, W, invW) - mulDivFloor(P.budget, C, W, invW);
                s = (uint32_t)(q < (unsigned long long)kSplitMax ? q : (unsigned long long)kSplitMax);
            }
            P.counts[t] = s;
        }
        carry += roundTotal;
        __syncthreads();
        uint32_t roundSplits;
        blockExclusive<uint32_t>(s, &roundSplits);
        __syncthreads();
        sum += roundSplits;
    }
    if (threadIdx.x == 0) {
        P.blockSums[chunk] = sum;
        if (sum) atomicAdd(P.totals + 1, (unsigned long long)sum);
    }
}

// Reference slots of triangles [b0, b1): each one's first slot (the references before
// it) and final split count, and its index on every slot it owns.
__device__ __forceinline__ void splitSlotsRange(const SplitParams& P, uint32_t chunk, uint32_t b0, uint32_t b1) {
    const unsigned long long given = __ldcg(P.totals + 1);
    const unsigned long long left = given < P.budget ? (unsigned long long)P.budget - given : 0ull;
    const uint32_t m = P.n + P.budget;
    uint32_t carry = __ldcg(P.blockSums + chunk);
    for (uint32_t base = b0; base < b1; base += blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        const uint32_t mine = t < b1 ? __ldcg(P.counts + t) : 0u;
        uint32_t roundTotal;
        const uint32_t local = blockExclusive<uint32_t>(mine, &roundTotal);
        if (t < b1) {
            const uint32_t extra = (unsigned long long)t < left ? 1u : 0u;
            const uint32_t first = t + carry + local + (uint32_t)((unsigned long long)t < left ? t : left);
            const uint32_t s = min(mine + extra, (uint32_t)kSplitMax + 1u);
            P.counts[t] = s;
            P.firstSlot[t] = first;
            for (uint32_t j = 0; j <= s; ++j) {
                if (first + j >= m) {  // cannot happen: the shares add up to at most the budget
                    latchError(P.error, GRT_ERROR_INTERNAL);
                    break;
                }
                P.slotTriangle[first + j] = t;
            }
        }
        carry += roundTotal;
        __syncthreads();
    }
}

// References [r0, r1), one thread each: the k-th leaf, left first, of its triangle's cut
// tree, found by walking down from the triangle's box and cutting only the boxes on its
// path (each cut as the depth-first order makes it); its box, triangle and owner flag,
// and with CENTROIDS its centroid and the centroid bounds (the batched launch takes
// those from its prep step instead).
template <bool CENTROIDS>
__device__ __forceinline__ void splitEmitRange(const SplitParams& P, uint32_t r0, uint32_t r1) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    const SplitGrid g = loadSplitGrid(P.sceneBounds);
    for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const uint32_t t = __ldcg(P.slotTriangle + r);
        uint32_t k = t < P.n ? r - __ldcg(P.firstSlot + t) : 0xFFFFFFFFu;
        int s = t < P.n ? (int)__ldcg(P.counts + t) : 0;
        if (t >= P.n || k > (uint32_t)s) {  // cannot happen; leave an empty reference of triangle 0
            latchError(P.error, GRT_ERROR_INTERNAL);
            P.refs[2 * (size_t)r] = make_float4(INFINITY, INFINITY, INFINITY, __uint_as_float(0u));
            P.refs[2 * (size_t)r + 1] = make_float4(-INFINITY, -INFINITY, -INFINITY, __uint_as_float(0u));
            continue;
        }
        float v[3][3];
        SBox cur;
        splitTriangle(P.src, t, v, &cur);
        const bool owner = k == 0;
        while (s > 0) {
            SBox L, R;
            int sL;
            cutOnce(g, v, cur, s, &L, &R, &sL);
            if (k <= (uint32_t)sL) {
                cur = L;
                s = sL;
            } else {
                cur = R;
                k -= (uint32_t)sL + 1u;
                s = s - 1 - sL;
            }
        }
        P.refs[2 * (size_t)r] = make_float4(cur.lo[0], cur.lo[1], cur.lo[2], __uint_as_float(t));
        P.refs[2 * (size_t)r + 1] = make_float4(cur.hi[0], cur.hi[1], cur.hi[2], __uint_as_float(owner ? 1u : 0u));
        if (CENTROIDS) {
            Box3 bb;
            bb.lo = make_float3(cur.lo[0], cur.lo[1], cur.lo[2]);
            bb.hi = make_float3(cur.hi[0], cur.hi[1], cur.hi[2]);
            const float3 c = boxCentroid(bb);
            P.centroids[r] = make_float4(c.x, c.y, c.z, 0.f);
            mn[0] = fminf(mn[0], c.x), mn[1] = fminf(mn[1], c.y), mn[2] = fminf(mn[2], c.z);
            mx[0] = fmaxf(mx[0], c.x), mx[1] = fmaxf(mx[1], c.y), mx[2] = fmaxf(mx[2], c.z);
        }
    }
    if (CENTROIDS) reduceBoxBounds(mn, mx, P.centroidBounds);
}

}  // namespace grt
