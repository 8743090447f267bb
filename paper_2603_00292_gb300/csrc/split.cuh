// Spatial splits of triangles before a build (GRT_BUILD_SPLIT_TRIANGLES): the paper's
// high-quality option names spatial splits (Sec. 8, SBVH); they are made here ahead of
// the build, after Karras and Aila ("Fast Parallel Construction of High-Quality Bounding
// Volume Hierarchies", HPG 2013): a budget S of extra references is shared out by a
// per-triangle priority, and each triangle is cut recursively at the most important
// plane of a 1024-cell grid over the scene that crosses its box. The build then runs
// over the n + S references (PrimSource kind 2) exactly as over primitives.
//
// Six launches, one thread per triangle where not said: the scene box; the weights
// (integer cube roots of the priority) and their per-block sums; one block's exclusive
// scan of those sums (and the total W); each triangle's share of the budget from its
// place in the running sum of weights, floor(S C_{t+1} / W) - floor(S C_t / W), and
// per-block sums of the shares; one block's scan of those; the cuts themselves, which
// write the references, their centroids and the centroid bounds. Every double operation
// is an explicit round-to-nearest intrinsic (nothing is fused), min / max are written
// as selections and the integer steps are exact, so the results are bit-for-bit those
// of any sequential IEEE-754 evaluation of the same steps.
#pragma once

#include "lbvh.cuh"

namespace grt {

constexpr int kSplitMax = 31;               // splits one triangle takes by priority (+1 from the remainder)
constexpr int kSplitStack = kSplitMax + 3;  // pending right sides of one triangle's cuts (<= its splits)
constexpr int kSplitThreads = 256;
constexpr int kSplitScanThreads = 1024;

struct SplitParams {
    PrimSource src;                // the triangles (idx / verts)
    uint32_t n;                    // triangles
    uint32_t budget;               // S
    uint32_t* sceneBounds;         // 6 ordered words: union of the triangle boxes
    unsigned long long* totals;    // [0] sum of the weights W, [1] splits handed out by priority
    uint32_t* counts;              // per triangle: its weight, then its priority splits
    unsigned long long* weightSums;  // per block of kSplitThreads triangles: weights, then their exclusive prefix
    uint32_t* blockSums;           // per block: splits, then their exclusive prefix
    uint32_t blocks;
    float4* refs;                  // (n + S) x {lo.xyz, triangle}, {hi.xyz, owner}
    float4* centroids;             // (n + S)
    uint32_t* centroidBounds;      // 6 ordered words
    uint32_t* error;               // device error word
};

struct SBox {
    float lo[3], hi[3];
};

__device__ __forceinline__ float selMin(float a, float b) { return b < a ? b : a; }
__device__ __forceinline__ float selMax(float a, float b) { return a < b ? b : a; }
__device__ __forceinline__ double dSelMax(double a, double b) { return a < b ? b : a; }

struct SplitGrid {
    double lo[3], ext[3], inv[3];
    float glo[3], ghi[3];
};

__device__ __forceinline__ SplitGrid loadSplitGrid(const uint32_t* b6) {
    SplitGrid g;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g.glo[a] = orderedToFloat(b6[a]);
        g.ghi[a] = orderedToFloat(b6[3 + a]);
        g.lo[a] = (double)g.glo[a];
        g.ext[a] = __dsub_rn((double)g.ghi[a], (double)g.glo[a]);
        g.inv[a] = g.ext[a] > 0.0 ? __ddiv_rn(1024.0, g.ext[a]) : 0.0;
    }
    return g;
}

// Cell of coordinate x on axis a: floor(q), or ceil(q) - 1 for the end of a box
// (a box ending on a grid line does not reach the next cell), clamped to [0, 1023].
__device__ __forceinline__ int gridCell(const SplitGrid& g, float x, int a, bool end) {
    if (g.inv[a] == 0.0) return 0;
    const double q = __dmul_rn(__dsub_rn((double)x, g.lo[a]), g.inv[a]);
    const double f = end ? __dsub_rn(ceil(q), 1.0) : floor(q);
    if (!(f >= 0.0)) return 0;
    if (f > 1023.0) return 1023;
    return (int)f;
}

// First and last cell of box b on axis a, the box narrowed by one float step at each end.
__device__ __forceinline__ void gridSpan(const SplitGrid& g, const SBox& b, int a, int* cl, int* ch) {
    *cl = gridCell(g, nextafterf(b.lo[a], INFINITY), a, false);
    const int e = gridCell(g, nextafterf(b.hi[a], -INFINITY), a, true);
    *ch = e > *cl ? e : *cl;
}

__device__ __forceinline__ int bitLength(uint32_t x) { return 32 - __clz(x); }

// Largest w with w^3 <= N (N <= 2^63): a double estimate, then exact integer steps.
__device__ __forceinline__ uint32_t integerCubeRoot(unsigned long long N) {
    unsigned long long w = (unsigned long long)cbrt((double)N);
    for (int i = 0; i < 4 && w > 0 && w * w * w > N; ++i) --w;
    for (int i = 0; i < 4 && (w + 1) * (w + 1) * (w + 1) <= N; ++i) ++w;
    return (uint32_t)w;
}

// floor(S X / W) exactly, for 0 < W < 2^63 and X <= W: a double estimate (off by at most
// one) corrected against the 128-bit product S X.
__device__ __forceinline__ unsigned long long mulDivFloor(uint32_t S, unsigned long long X, unsigned long long W) {
    const unsigned long long ph = __umul64hi((unsigned long long)S, X), pl = (unsigned long long)S * X;
    unsigned long long q = (unsigned long long)floor(__ddiv_rn(__dmul_rn((double)S, (double)X), (double)W));
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

__device__ __forceinline__ double halfArea(const SBox& b) {
    const double dx = __dsub_rn((double)b.hi[0], (double)b.lo[0]);
    const double dy = __dsub_rn((double)b.hi[1], (double)b.lo[1]);
    const double dz = __dsub_rn((double)b.hi[2], (double)b.lo[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dy), __dmul_rn(dy, dz)), __dmul_rn(dz, dx));
}

__device__ __forceinline__ double longestExtent(const SBox& b) {
    double w = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) w = dSelMax(w, __dsub_rn((double)b.hi[a], (double)b.lo[a]));
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

// The cutting plane of box b: the grid line of the highest level strictly inside it
// (ties: longer extent, then lower axis), else the midpoint of its longest axis.
__device__ __forceinline__ void cutPlane(const SplitGrid& g, const SBox& b, int* axis, float* plane) {
    int best = -1, bestBit = -1, bestJ = 0;
    double bestExt = -1.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int cl, ch;
        gridSpan(g, b, a, &cl, &ch);
        if (cl == ch) continue;
        const int bit = bitLength((uint32_t)(cl ^ ch)) - 1;
        const double e = __dsub_rn((double)b.hi[a], (double)b.lo[a]);
        if (bit > bestBit || (bit == bestBit && e > bestExt)) best = a, bestBit = bit, bestExt = e, bestJ = (ch >> bit) << bit;
    }
    if (best >= 0) {
        *axis = best;
        *plane = __double2float_rn(__dadd_rn(g.lo[best], __dmul_rn((double)bestJ, __dmul_rn(g.ext[best], 1.0 / 1024.0))));
        return;
    }
    int a0 = 0;
    double e0 = __dsub_rn((double)b.hi[0], (double)b.lo[0]);
#pragma unroll
    for (int a = 1; a < 3; ++a) {
        const double e = __dsub_rn((double)b.hi[a], (double)b.lo[a]);
        if (e > e0) a0 = a, e0 = e;
    }
    *axis = a0;
    *plane = __double2float_rn(__dmul_rn(0.5, __dadd_rn((double)b.lo[a0], (double)b.hi[a0])));
}

// Box of the triangle's part on one side of x_axis = P (vertices on that side, edge
// crossings widened by 2^-47 of the endpoint magnitude and rounded outward), within b.
__device__ __forceinline__ SBox clipSide(const float v[3][3], int axis, float P, bool left, const SBox& b) {
    SBox r;
#pragma unroll
    for (int c = 0; c < 3; ++c) r.lo[c] = INFINITY, r.hi[c] = -INFINITY;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool in = left ? v[i][axis] <= P : v[i][axis] >= P;
        if (!in) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) r.lo[c] = selMin(r.lo[c], v[i][c]), r.hi[c] = selMax(r.hi[c], v[i][c]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float* a = v[i];
        const float* e = v[i == 2 ? 0 : i + 1];
        const bool crosses = (a[axis] < P && e[axis] > P) || (a[axis] > P && e[axis] < P);
        if (!crosses) continue;
        const double t = __ddiv_rn(__dsub_rn((double)P, (double)a[axis]), __dsub_rn((double)e[axis], (double)a[axis]));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c == axis) {
                r.lo[c] = selMin(r.lo[c], P), r.hi[c] = selMax(r.hi[c], P);
                continue;
            }
            const double q = __dadd_rn((double)a[c], __dmul_rn(__dsub_rn((double)e[c], (double)a[c]), t));
            const double pad = __dmul_rn(dSelMax(fabs((double)a[c]), fabs((double)e[c])), 0x1p-47);
            r.lo[c] = selMin(r.lo[c], __double2float_rd(__dsub_rn(q, pad)));
            r.hi[c] = selMax(r.hi[c], __double2float_ru(__dadd_rn(q, pad)));
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) r.lo[c] = selMax(r.lo[c], b.lo[c]), r.hi[c] = selMin(r.hi[c], b.hi[c]);
    return r;
}

// ----------------------------------------------------------------------- kernels
__global__ void __launch_bounds__(kSplitThreads) splitBoundsKernel(SplitParams P) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (t < P.n) {
        float v[3][3];
        SBox b;
        splitTriangle(P.src, t, v, &b);
        for (int a = 0; a < 3; ++a) mn[a] = b.lo[a], mx[a] = b.hi[a];
    }
    reduceBoxBounds(mn, mx, P.sceneBounds);
}

// Exclusive prefix of x over the block (kSplitThreads threads), and the block's total.
template <typename T>
__device__ __forceinline__ T blockExclusive(T x, T* total) {
    __shared__ T warpSums[kSplitThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warpSums[warp] = inc;
    __syncthreads();
    T before = inc - x, all = 0;
    for (int w = 0; w < kSplitThreads / 32; ++w) {
        if (w < warp) before += warpSums[w];
        all += warpSums[w];
    }
    *total = all;
    return before;
}

__global__ void __launch_bounds__(kSplitThreads) splitWeightKernel(SplitParams P) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t w = 0;
    if (t < P.n) {
        const SplitGrid g = loadSplitGrid(P.sceneBounds);
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
        double e1[3], e2[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            e1[a] = __dsub_rn((double)v[1][a], (double)v[0][a]);
            e2[a] = __dsub_rn((double)v[2][a], (double)v[0][a]);
        }
        const double cx = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
        const double cy = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
        const double cz = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
        const double tri = __dmul_rn(0.5, __dadd_rn(__dadd_rn(fabs(cx), fabs(cy)), fabs(cz)));
        double excess = __dsub_rn(halfArea(b), tri);
        if (!(excess > 0.0)) excess = 0.0;
        SBox G;
        for (int a = 0; a < 3; ++a) G.lo[a] = g.glo[a], G.hi[a] = g.ghi[a];
        const double areaG = halfArea(G);
        const double r = areaG > 0.0 ? __dmul_rn(__ddiv_rn(excess, areaG), (double)(1u << level)) : 0.0;
        w = integerCubeRoot((unsigned long long)__dmul_rn(r, 9007199254740992.0));  // r 2^53
        P.counts[t] = w;
    }
    unsigned long long total;
    blockExclusive<unsigned long long>(w, &total);
    if (threadIdx.x == 0) P.weightSums[blockIdx.x] = total;
}

// One block: exclusive prefix sums of `count` per-block values, in place; the total
// goes to *total.
template <typename T>
__device__ __forceinline__ void scanBlockSums(T* v, uint32_t count, unsigned long long* total) {
    __shared__ T warpSums[kSplitScanThreads / 32];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < count; base += kSplitScanThreads) {
        const uint32_t i = base + threadIdx.x;
        const T x = i < count ? v[i] : (T)0;
        T inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warpSums[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            T ws = warpSums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T y = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += y;
            }
            warpSums[lane] = ws;  // inclusive over warps
        }
        __syncthreads();
        const T before = carry + (warp ? warpSums[warp - 1] : (T)0) + inc - x;
        if (i < count) v[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += warpSums[kSplitScanThreads / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = (unsigned long long)carry;
}

__global__ void __launch_bounds__(kSplitScanThreads) splitScanWeightsKernel(SplitParams P) {
    scanBlockSums<unsigned long long>(P.weightSums, P.blocks, P.totals);
}

// Triangle t's splits by priority: its share of the budget between the running weight
// sums before and after it, capped at kSplitMax.
__global__ void __launch_bounds__(kSplitThreads) splitCountKernel(SplitParams P) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long w = t < P.n ? P.counts[t] : 0ull;
    unsigned long long blockTotal;
    const unsigned long long local = blockExclusive<unsigned long long>(w, &blockTotal);
    uint32_t s = 0;
    if (t < P.n) {
        const unsigned long long W = P.totals[0];
        if (W) {
            const unsigned long long C = P.weightSums[blockIdx.x] + local;
            const unsigned long long q = mulDivFloor(P.budget, C + w, W) - mulDivFloor(P.budget, C, W);
            s = (uint32_t)(q < (unsigned long long)kSplitMax ? q : (unsigned long long)kSplitMax);
        }
        P.counts[t] = s;
    }
    __syncthreads();  // the block's shared partial sums are reused below
    uint32_t sum;
    blockExclusive<uint32_t>(s, &sum);
    if (threadIdx.x == 0) {
        P.blockSums[blockIdx.x] = sum;
        if (sum) atomicAdd(P.totals + 1, (unsigned long long)sum);
    }
}

__global__ void __launch_bounds__(kSplitScanThreads) splitScanKernel(SplitParams P) {
    scanBlockSums<uint32_t>(P.blockSums, P.blocks, nullptr);
}

__device__ __forceinline__ void emitRef(const SplitParams& P, uint32_t slot, const SBox& b, uint32_t t, bool owner,
                                        float mn[3], float mx[3]) {
    if (slot >= P.n + P.budget) {  // cannot happen: the shares add up to at most the budget
        latchError(P.error, GRT_ERROR_INTERNAL);
        return;
    }
    P.refs[2 * (size_t)slot] = make_float4(b.lo[0], b.lo[1], b.lo[2], __uint_as_float(t));
    P.refs[2 * (size_t)slot + 1] = make_float4(b.hi[0], b.hi[1], b.hi[2], __uint_as_float(owner ? 1u : 0u));
    Box3 bb;
    bb.lo = make_float3(b.lo[0], b.lo[1], b.lo[2]);
    bb.hi = make_float3(b.hi[0], b.hi[1], b.hi[2]);
    const float3 c = boxCentroid(bb);
    P.centroids[slot] = make_float4(c.x, c.y, c.z, 0.f);
    mn[0] = fminf(mn[0], c.x), mn[1] = fminf(mn[1], c.y), mn[2] = fminf(mn[2], c.z);
    mx[0] = fmaxf(mx[0], c.x), mx[1] = fmaxf(mx[1], c.y), mx[2] = fmaxf(mx[2], c.z);
}

__global__ void __launch_bounds__(kSplitThreads) splitEmitKernel(SplitParams P) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t mine = t < P.n ? P.counts[t] : 0u;
    uint32_t blockTotal;
    const uint32_t local = blockExclusive<uint32_t>(mine, &blockTotal);
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (t < P.n) {
        const unsigned long long given = P.totals[1];
        const unsigned long long left = given < P.budget ? (unsigned long long)P.budget - given : 0ull;
        const uint32_t extra = (unsigned long long)t < left ? 1u : 0u;
        uint32_t slot = t + P.blockSums[blockIdx.x] + local + (uint32_t)((unsigned long long)t < left ? t : left);
        const SplitGrid g = loadSplitGrid(P.sceneBounds);
        float v[3][3];
        SBox cur;
        splitTriangle(P.src, t, v, &cur);
        int s = (int)min(mine + extra, (uint32_t)kSplitMax + 1u);  // keeps the pending stack in bounds
        SBox pendBox[kSplitStack];
        int pendS[kSplitStack];
        int sp = 0;
        bool owner = true;
        for (;;) {
            if (s == 0) {
                emitRef(P, slot++, cur, t, owner, mn, mx);
                owner = false;
                if (sp == 0) break;
                --sp;
                cur = pendBox[sp];
                s = pendS[sp];
                continue;
            }
            int axis;
            float plane;
            cutPlane(g, cur, &axis, &plane);
            SBox L = clipSide(v, axis, plane, true, cur), R = clipSide(v, axis, plane, false, cur);
            const int rest = s - 1;
            int sL;
            const bool eL = boxEmpty(L), eR = boxEmpty(R);
            if (eL && eR) {
                L = R = cur;
                sL = 0;
            } else if (eL) {
                L = R;
                sL = 0;
            } else if (eR) {
                R = L;
                sL = rest;
            } else {
                const double wL = longestExtent(L), wR = longestExtent(R);
                const double sum = __dadd_rn(wL, wR);
                sL = sum > 0.0 ? (int)floor(__dadd_rn(__ddiv_rn(__dmul_rn((double)rest, wL), sum), 0.5)) : rest / 2;
                sL = sL < rest ? sL : rest;
            }
            pendBox[sp] = R;  // s strictly decreases down every path, so sp stays below kSplitStack
            pendS[sp] = rest - sL;
            ++sp;
            cur = L;
            s = sL;
        }
    }
    reduceBoxBounds(mn, mx, P.centroidBounds);
}

}  // namespace grt
