// Device traversal core shared by the trace, ambient-occlusion, shading and batched
// kernels.
//
// Method: stack-based BVH traversal (paper Sec. 6.2 "BVH Traversal") through a
// two-level hierarchy whose instance leaves take the ray to object space with the
// inverse frame (Sec. 6.2 "Two-Level Hierarchy and Instancing"); the stack keeps its
// first entries in shared memory and spills to a global buffer (Sec. 7.5); closest-
// hit and any-hit queries (Sec. 7.5; any-hit may stop at the first valid hit, Sec.
// 4.2); custom primitives through a (ray type x geometry type) function table (Sec.
// 7.4). Triangles: Moller-Trumbore (1997), double-sided with inclusive edges as the
// paper's test (Sec. 3.1). Spheres: centre-relative discriminant of Haines et al.,
// "Precision Improvements for Ray/Sphere Intersection" (Ray Tracing Gems, 2019).
//
// Precision design. Decisions are taken in float32 with certified error bounds:
//  * box tests use the far-distance factor 1 + 2*gamma_3 of Ize, "Robust BVH Ray
//    Traversal" (JCGT 2013), near/far planes chosen by the direction's sign so that a
//    0*inf = NaN is dropped conservatively, and boxes are widened by the bound on the
//    object-space ray's transform error;
//  * a triangle or sphere test whose float32 edge functions (or discriminant) lie
//    within their rounding bound of zero is decided again in FP64;
//  * the closest hit's t, u, v are recomputed once in double-float arithmetic (refineFF).
// FP64 runs far slower than FP32 on this GPU, so it is confined to these rare cases.
#pragma once

#include <type_traits>

#include "grt_internal.cuh"

namespace grt {

constexpr uint32_t kSentinel = 0xFFFFFFFEu;  // stack marker: leave the current instance
constexpr uint32_t kNone = 0xFFFFFFFFu;
// Node formats a walk may meet, as a template argument (FM): 0 = 4-wide nodes only;
// 1 = 4-wide or quantised, read per level; 2 = 8-wide nodes (kWide8Words float4) on
// every level; 3 = any of the three, read per level (user kernels, which cannot know).
// W(FM) = slots per visit.
constexpr int kFmPlain = 0, kFmQuant = 1, kFmWide8 = 2, kFmMixed = 3;
__host__ __device__ constexpr int slotsOf(int fm) { return (fm & 2) ? 8 : 4; }
// queued leaves per lane (phased traversal): a node visit may queue W more while at most
// 4 are pending
__host__ __device__ constexpr uint32_t pendingCap(int w) { return w == 8 ? 12u : 8u; }
// Shared memory per thread of a kernel that runs refillLoop, in words: its stack slice
// of `depth` entries and its queue of pending leaves.
__host__ __device__ constexpr uint32_t traceSmemWords(uint32_t depth, int w = 4) { return depth + pendingCap(w); }
constexpr float kEps = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of float32
// 1 + 2*gamma(3) rounded up, gamma(n) = n*eps/(1 - n*eps)
constexpr float kFarScale = 1.0000005f;
// coefficients of the rounding terms of the triangle and sphere error bounds (see
// triangleTest and sphereTest)
constexpr float kBound = 8.0f * kEps;
constexpr float kSphereBound = 24.0f * kEps;

struct TraceTarget {
    const float4* nodes;  // top-level nodes (scene) or the geometry's nodes
    const void* leaves;
    uint32_t primType;  // of the geometry when tracing one directly
    uint32_t geomType;
    uint32_t empty;
    uint32_t fmt;  // node format: 0 4-wide (kWideWords float4), 1 quantised 4-wide (kQuantWords), 2 8-wide
    uint32_t split;  // a geometry whose triangles are split over several leaves
};

struct TraceParams {
    TraceTarget target;
    const float4* rays;  // 2 float4 per ray
    uint32_t* hits;      // 5 words per ray
    uint32_t count;
    const FuncEntry* table;
    uint32_t numGeomTypes;
    uint32_t rayType;
    uint32_t sharedDepth;
    uint32_t globalDepth;
    uint32_t* globalStack;  // [entry][thread]
    uint32_t globalStride;  // threads in the grid
    unsigned long long* counter;
    uint32_t* error;
    uint32_t maxSteps;
    uint32_t refillBelow;           // refill a warp when at most this many lanes hold a ray
    uint32_t rayMask;               // instances whose mask shares no bit with it are skipped
    const InstanceFrames64* inv64;  // scene: FP64 inverse frames by instance ID
    unsigned long long* stats;      // counting variants: grtTraceStatistics sums
    // fused ambient occlusion
    const float4* primaryRays;
    const uint32_t* primaryHits;
    const InstanceRecord* sceneLeaves;
    const uint32_t* scenePrimToLeaf;
    const uint32_t* targetPrimToLeaf;  // a triangle geometry traced directly: primitive ID -> leaf
    const float4* fwd32;
    uint32_t spp;
    unsigned long long seed;
    float aoLength;
    float* ao;
};

struct Hit {
    uint32_t inst, prim;
    float t, u, v;
};

// No user functions: the library's own kernels trace with this (the user branches
// compile away). A user kernel tracing through grt_device.cuh may pass a functor U with
//   bool intersect(uint32_t func, const grtRay& ray, const void* data, void* payload, grtHit& hit) const
//   bool filter(uint32_t func, const grtRay& ray, const void* data, void* payload, const grtHit& hit) const
// called for table entries naming user intersectors (func >= GRT_INTERSECT_USER) and
// user filters (>= GRT_FILTER_USER); see grt_device.cuh.
struct NoUser {};
template <class U>
constexpr bool kHasUser = !std::is_same<U, NoUser>::value;

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float norm1(float3 a) { return fabsf(a.x) + fabsf(a.y) + fabsf(a.z); }
__device__ __forceinline__ float3 normalize3(float3 a) {
    const float l = sqrtf(dot3(a, a));
    return make_float3(a.x / l, a.y / l, a.z / l);
}

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(float3 a) { return D3{(double)a.x, (double)a.y, (double)a.z}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dotd(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 crossd(D3 a, D3 b) {
    return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Ray state at the current level. The level's origin o sits at world parameter tOff,
// so a local parameter t' on this level is the world parameter tOff + t'.
struct Level {
    float3 o, d, id;  // float32 ray and reciprocal direction
    float3 on, of;    // origins for the near and far slab planes (box widening applied)
    float dO, dD;     // bounds on the error of each origin / direction component
    float dl1;        // |d|_1
    float tOff;       // world parameter of o
};

__device__ __forceinline__ void exactLevel(Level& L, float3 o, float3 d) {
    L.o = o;
    L.d = d;
    L.id = make_float3(__frcp_rn(d.x), __frcp_rn(d.y), __frcp_rn(d.z));
    L.on = o;
    L.of = o;
    L.dO = 0.f;
    L.dD = 0.f;
    L.dl1 = norm1(d);
    L.tOff = 0.f;
}

// World parameter range [a, b] as a local range on level L, widened by the rounding of
// the subtraction.
__device__ __forceinline__ float localLo(const Level& L, float a) {
    return L.tOff == 0.f ? a : (a - L.tOff) - kEps * (fabsf(a) + fabsf(L.tOff));
}
__device__ __forceinline__ float localHi(const Level& L, float b) {
    return L.tOff == 0.f ? b : (b - L.tOff) + kEps * (fabsf(b) + fabsf(L.tOff));
}

// Slab test of the four slots of wide node w. Per axis the near plane is the slot's lo
// for a non-negative direction (else hi) and its distance (p - on) * id; the far plane
// likewise with of. A slot is hit when the largest near distance (and tmin) is at most
// the smallest far distance (and tmax) times Ize's far factor. Returns the mask of
// slots hit; tn gets each slot's entry distance and c its child word. Empty slots
// (child kNone) never count as hit.
__device__ __forceinline__ uint32_t slab4(const float4* nodes, uint32_t w, const Level& L, float tmin, float tmax,
                                          float tn[4], uint32_t c[4]) {
    const float4* W = nodes + kWideWords * (size_t)w;
    // near and far planes of each axis: lo for a non-negative direction, else hi
    const uint32_t sx = L.id.x >= 0.f ? 0u : 1u, sy = L.id.y >= 0.f ? 0u : 1u, sz = L.id.z >= 0.f ? 0u : 1u;
    const float4 nx = __ldg(W + sx), fx = __ldg(W + (1u - sx));
    const float4 ny = __ldg(W + 2 + sy), fy = __ldg(W + 2 + (1u - sy));
    const float4 nz = __ldg(W + 4 + sz), fz = __ldg(W + 4 + (1u - sz));
    const float4 cw = __ldg(W + 6);
    const float px[4] = {nx.x, nx.y, nx.z, nx.w}, qx[4] = {fx.x, fx.y, fx.z, fx.w};
    const float py[4] = {ny.x, ny.y, ny.z, ny.w}, qy[4] = {fy.x, fy.y, fy.z, fy.w};
    const float pz[4] = {nz.x, nz.y, nz.z, nz.w}, qz[4] = {fz.x, fz.y, fz.z, fz.w};
    c[0] = __float_as_uint(cw.x), c[1] = __float_as_uint(cw.y), c[2] = __float_as_uint(cw.z), c[3] = __float_as_uint(cw.w);
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        tn[j] = fmaxf(fmaxf((px[j] - L.on.x) * L.id.x, (py[j] - L.on.y) * L.id.y),
                      fmaxf((pz[j] - L.on.z) * L.id.z, tmin));
        const float tf = fminf(fminf((qx[j] - L.of.x) * L.id.x, (qy[j] - L.of.y) * L.id.y),
                               fminf((qz[j] - L.of.z) * L.id.z, tmax));
        if (tn[j] <= tf * kFarScale && c[j] != kInvalid) m |= 1u << j;
    }
    return m;
}

// Byte j of w as a float: the byte becomes the low mantissa bits of 2^23, which is then
// subtracted (exact).
__device__ __forceinline__ float byteToFloat(uint32_t w, uint32_t j) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7650u | j)) - 8388608.0f;
}

// slab4 for a quantised 4-wide node (kQuantWords float4: origin p.xyz and the biased
// exponents; the lower and upper plane bytes of each axis; the child words). Each plane
// the test uses is decoded as fl(p + q 2^e) (one FMA: q 2^e is exact), which is the box
// the build made sure contains the child's box, and then tested exactly as in slab4.
__device__ __forceinline__ uint32_t slab4q(const float4* nodes, uint32_t w, const Level& L, float tmin, float tmax,
                                           float tn[4], uint32_t c[4]) {
    const float4* Q = nodes + kQuantWords * (size_t)w;
    const float4 h = __ldg(Q), a = __ldg(Q + 1), b = __ldg(Q + 2), d = __ldg(Q + 3);
    const uint32_t ew = __float_as_uint(h.w);
    const float sx = __uint_as_float((ew & 0xFFu) << 23), sy = __uint_as_float(((ew >> 8) & 0xFFu) << 23),
                sz = __uint_as_float(((ew >> 16) & 0xFFu) << 23);
    const bool px = L.id.x >= 0.f, py = L.id.y >= 0.f, pz = L.id.z >= 0.f;
    const uint32_t nxw = __float_as_uint(px ? a.x : a.y), fxw = __float_as_uint(px ? a.y : a.x);
    const uint32_t nyw = __float_as_uint(py ? a.z : a.w), fyw = __float_as_uint(py ? a.w : a.z);
    const uint32_t nzw = __float_as_uint(pz ? b.x : b.y), fzw = __float_as_uint(pz ? b.y : b.x);
    c[0] = __float_as_uint(b.z), c[1] = __float_as_uint(b.w), c[2] = __float_as_uint(d.x), c[3] = __float_as_uint(d.y);
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float nx = __fmaf_rn(byteToFloat(nxw, j), sx, h.x), fx = __fmaf_rn(byteToFloat(fxw, j), sx, h.x);
        const float ny = __fmaf_rn(byteToFloat(nyw, j), sy, h.y), fy = __fmaf_rn(byteToFloat(fyw, j), sy, h.y);
        const float nz = __fmaf_rn(byteToFloat(nzw, j), sz, h.z), fz = __fmaf_rn(byteToFloat(fzw, j), sz, h.z);
        tn[j] = fmaxf(fmaxf((nx - L.on.x) * L.id.x, (ny - L.on.y) * L.id.y), fmaxf((nz - L.on.z) * L.id.z, tmin));
        const float tf =
            fminf(fminf((fx - L.of.x) * L.id.x, (fy - L.of.y) * L.id.y), fminf((fz - L.of.z) * L.id.z, tmax));
        if (tn[j] <= tf * kFarScale && c[j] != kInvalid) m |= 1u << j;
    }
    return m;
}

// Slab test of the eight slots of 8-wide node w (kWide8Words float4): rows 4a + 2 side
// + half hold axis a's lower (side 0) or upper (side 1) planes of slots 4 half .. 4 half
// + 3, rows 12 and 13 the child words. The same certified test as slab4, per slot.
__device__ __forceinline__ uint32_t slab8(const float4* nodes, uint32_t w, const Level& L, float tmin, float tmax,
                                          float tn[8], uint32_t c[8]) {
    const float4* N = nodes + kWide8Words * (size_t)w;
    const uint32_t sx = L.id.x >= 0.f ? 0u : 2u, sy = L.id.y >= 0.f ? 0u : 2u, sz = L.id.z >= 0.f ? 0u : 2u;
    uint32_t m = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float4 nx = __ldg(N + sx + h), fx = __ldg(N + (2u - sx) + h);
        const float4 ny = __ldg(N + 4 + sy + h), fy = __ldg(N + 4 + (2u - sy) + h);
        const float4 nz = __ldg(N + 8 + sz + h), fz = __ldg(N + 8 + (2u - sz) + h);
        const float4 cw = __ldg(N + 12 + h);
        const float px[4] = {nx.x, nx.y, nx.z, nx.w}, qx[4] = {fx.x, fx.y, fx.z, fx.w};
        const float py[4] = {ny.x, ny.y, ny.z, ny.w}, qy[4] = {fy.x, fy.y, fy.z, fy.w};
        const float pz[4] = {nz.x, nz.y, nz.z, nz.w}, qz[4] = {fz.x, fz.y, fz.z, fz.w};
        const uint32_t cc[4] = {__float_as_uint(cw.x), __float_as_uint(cw.y), __float_as_uint(cw.z),
                                __float_as_uint(cw.w)};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = 4 * h + j;
            c[k] = cc[j];
            tn[k] = fmaxf(fmaxf((px[j] - L.on.x) * L.id.x, (py[j] - L.on.y) * L.id.y),
                          fmaxf((pz[j] - L.on.z) * L.id.z, tmin));
            const float tf = fminf(fminf((qx[j] - L.of.x) * L.id.x, (qy[j] - L.of.y) * L.id.y),
                                   fminf((qz[j] - L.of.z) * L.id.z, tmax));
            if (tn[k] <= tf * kFarScale && cc[j] != kInvalid) m |= 1u << k;
        }
    }
    return m;
}

__device__ __forceinline__ uint32_t pick4(const uint32_t c[4], uint32_t j) {
    return j == 0 ? c[0] : j == 1 ? c[1] : j == 2 ? c[2] : c[3];
}

// Float32 Moller-Trumbore with certified bounds on the three edge values.
// Returns 0 = miss, 1 = hit with world t in [tmin, tmax] (t, u, v set), 2 = undecided
// in float32. Rounding bound: T, e2 and the cross product each contribute at most u
// times their magnitude and the dot product 3u, so |U - U*| <= 7u * sum|T_i|(|d_j||e2_k|
// + |d_k||e2_j|) <= 7u * |T|_1 |d|_1 |e2|_1 (likewise for V and det); kBound = 8u.
__device__ __forceinline__ int triangleTest(const Level& L, float3 v0, float3 v1, float3 v2, float e1n, float e2n,
                                           float tmin, float tmax, bool strict, float& t, float& u, float& v) {
    const float3 e1 = v1 - v0, e2 = v2 - v0;
    const float3 P = cross3(L.d, e2);
    const float det = dot3(e1, P);
    const float ad = fabsf(det);
    const float Edet = (4.f * L.dD + kBound * L.dl1) * e1n * e2n;
    if (ad <= Edet) return (ad == 0.f && Edet == 0.f) ? 0 : 2;
    const float s = det > 0.f ? 1.f : -1.f;
    const float3 T = L.o - v0;
    const float Tn = norm1(T);
    const float U = dot3(T, P) * s;
    const float EU = 2.f * (L.dO * norm1(P) + 2.f * L.dD * Tn * e2n) + kBound * Tn * L.dl1 * e2n;
    if (U < -EU) return 0;
    const float3 Q = cross3(T, e1);
    const float V = dot3(L.d, Q) * s;
    const float EV = 4.f * (L.dO * L.dl1 + L.dD * Tn) * e1n + kBound * Tn * L.dl1 * e1n;
    if (V < -EV) return 0;
    const float W = ad - U - V;
    const float EW = Edet + EU + EV + 4.f * kEps * (ad + fabsf(U) + fabsf(V));
    if (W < -EW) return 0;
    if (U <= EU || V <= EV || W <= EW) return 2;
    t = dot3(e2, Q) / det + L.tOff;
    u = U / ad;
    v = V / ad;
    return (t >= tmin && (strict ? t < tmax : t <= tmax)) ? 1 : 0;
}

// FP64 Moller-Trumbore with the same acceptance rules (u in [0,1], v >= 0, u+v <= 1).
__device__ __forceinline__ bool triangleTest64(D3 o, D3 d, float3 v0f, float3 v1f, float3 v2f, double tmin, double tmax,
                                            bool strict, double& t, double& u, double& v) {
    const D3 v0 = d3(v0f), e1 = d3(v1f) - v0, e2 = d3(v2f) - v0;
    const D3 P = crossd(d, e2);
    const double det = dotd(e1, P);
    if (det == 0.0) return false;
    const double inv = 1.0 / det;
    const D3 T = o - v0;
    u = dotd(T, P) * inv;
    if (u < 0.0 || u > 1.0) return false;
    const D3 Q = crossd(T, e1);
    v = dotd(d, Q) * inv;
    if (v < 0.0 || u + v > 1.0) return false;
    t = dotd(e2, Q) * inv;
    return t >= tmin && (strict ? t < tmax : t <= tmax);
}

// FP64 barycentrics and distance of a known hit (no acceptance test).

// Float32 sphere test. Returns 0 = miss, 1 = hit (world t set), 2 = undecided.
__device__ __forceinline__ int sphereTest(const Level& L, const float4& s, float tmin, float tmax, bool strict, float& t) {
    const float3 f = L.o - make_float3(s.x, s.y, s.z);
    const float a = dot3(L.d, L.d);
    if (a == 0.f) return L.dD > 0.f ? 2 : 0;
    const float b = dot3(f, L.d);
    const float tca = b / a;
    const float3 l = f - L.d * tca;
    const float r2 = s.w * s.w;
    const float D = r2 - dot3(l, l);
    const float fn = dot3(f, f);
    // position error at the closest approach, then its effect on r^2 - |l|^2
    const float ep = 1.7320508f * (L.dO + fabsf(tca) * L.dD);
    const float E = kSphereBound * (fn + r2) + 4.f * sqrtf(fn) * ep + ep * ep;
    if (D < -E) return 0;
    if (D <= E) return 2;
    const float c = fn - r2;
    const float q = -b - copysignf(sqrtf(a * D), b);
    float t0 = ((q != 0.0f) ? c / q : 0.0f) + L.tOff;
    float t1 = q / a + L.tOff;
    if (t0 > t1) {
        const float x = t0;
        t0 = t1;
        t1 = x;
    }
    // roots near the ray's range ends are left to the undecided path
    const float et = 8.f * kEps * (fabsf(t0) + fabsf(t1)) + 4.f * ep / sqrtf(a);
    if (fabsf(t0 - tmin) <= et || fabsf(t1 - tmin) <= et) return 2;
    if (t0 >= tmin && (strict ? t0 < tmax : t0 <= tmax)) {
        t = t0;
        return 1;
    }
    if (t1 >= tmin && (strict ? t1 < tmax : t1 <= tmax)) {
        t = t1;
        return 1;
    }
    return 0;
}

// FP64 sphere: smallest root of |o + t d - c|^2 = r^2 in range.
__device__ __forceinline__ bool sphereTest64(D3 o, D3 d, float4 s, double tmin, double tmax, bool strict, double& t) {
    const D3 f = o - D3{(double)s.x, (double)s.y, (double)s.z};
    const double a = dotd(d, d);
    const double b = dotd(f, d);
    const double rr = (double)s.w * (double)s.w;
    const double c = dotd(f, f) - rr;
    const double disc = b * b - a * c;
    if (disc < 0.0 || a == 0.0) return false;
    const double sq = sqrt(disc);
    const double t0 = (-b - sq) / a, t1 = (-b + sq) / a;
    if (t0 >= tmin && (strict ? t0 < tmax : t0 <= tmax)) {
        t = t0;
        return true;
    }
    if (t1 >= tmin && (strict ? t1 < tmax : t1 <= tmax)) {
        t = t1;
        return true;
    }
    return false;
}

// FP64 ray at the current level: the world ray itself, or its image under the
// instance's FP64 inverse frame.
__device__ __forceinline__ void ray64(const InstanceFrames64* inv64, bool inInstance, uint32_t inst, float3 wo, float3 wd,
                                      D3& o, D3& d) {
    if (!inInstance) {
        o = d3(wo);
        d = d3(wd);
        return;
    }
    const InstanceFrames64& F = inv64[inst];
    double r[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r[k] = F.inv[k][0] * (double)wo.x + F.inv[k][1] * (double)wo.y + F.inv[k][2] * (double)wo.z + F.inv[k][3];
        r[3 + k] = F.inv[k][0] * (double)wd.x + F.inv[k][1] * (double)wd.y + F.inv[k][2] * (double)wd.z;
    }
    o = D3{r[0], r[1], r[2]};
    d = D3{r[3], r[4], r[5]};
}

// FP64 decision of a primitive test that float32 could not take, kept out of line
// (and value-in, value-out) so that it weighs neither on the traversal loop's
// registers nor on its memory. Returns (t, u, v, 1) for a hit, w = 0 for a miss.
static __device__ __noinline__ float4 decide64(const InstanceFrames64* inv64, bool inInstance, uint32_t inst, float3 wo,
                                        float3 wd, const float4* rec, bool sphere, float tmin, float tmax,
                                        bool strict) {
    D3 o, d;
    ray64(inv64, inInstance, inst, wo, wd, o, d);
    if (sphere) {
        double t64;
        if (!sphereTest64(o, d, __ldg(rec), tmin, tmax, strict, t64)) return make_float4(0.f, 0.f, 0.f, 0.f);
        return make_float4((float)t64, 0.f, 0.f, 1.f);
    }
    double t64, u64, v64;
    if (!triangleTest64(o, d, f3(__ldg(rec)), f3(__ldg(rec + 1)), f3(__ldg(rec + 2)), tmin, tmax, strict, t64, u64,
                        v64))
        return make_float4(0.f, 0.f, 0.f, 0.f);
    return make_float4((float)t64, (float)u64, (float)v64, 1.f);
}

// Error-free transformations (Dekker; Knuth): a*b = p + e and a + b = s + e exactly.
__device__ __forceinline__ float2 twoProd(float a, float b) {
    const float p = __fmul_rn(a, b);
    return make_float2(p, fmaf(a, b, -p));
}
__device__ __forceinline__ float2 twoSum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// Object-space point of the world ray at world parameter te, from the inverse frame
// held as float32 rows plus low parts (hi + lo = the FP64 frame to 2^-48), evaluated
// in float-float arithmetic (about 48 significant bits) and rounded to float32. This
// stays on the float32 pipes: FP64 is far slower on this GPU.
__device__ __forceinline__ float3 instanceOriginFF(const float4* hi, const float4* lo, float3 wo, float3 wd, float te) {
    const float wo3[3] = {wo.x, wo.y, wo.z}, wd3[3] = {wd.x, wd.y, wd.z};
    float wh[3], wl[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // w = wo + te * wd as hi + lo
        const float2 p = twoProd(te, wd3[j]);
        const float2 q = twoSum(wo3[j], p.x);
        wh[j] = q.x;
        wl[j] = __fadd_rn(q.y, p.y);
    }
    float o[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 H = __ldg(hi + k), Lw = __ldg(lo + k);
        const float gh[3] = {H.x, H.y, H.z}, gl[3] = {Lw.x, Lw.y, Lw.z};
        float ah = H.w, al = Lw.w;  // translation part
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float2 p = twoProd(gh[j], wh[j]);
            const float pl = fmaf(gh[j], wl[j], fmaf(gl[j], wh[j], p.y));
            const float2 q = twoSum(ah, p.x);
            ah = q.x;
            al = __fadd_rn(al, __fadd_rn(q.y, pl));
        }
        o[k] = __fadd_rn(ah, al);
    }
    return make_float3(o[0], o[1], o[2]);
}

// ---------------------------------------------------------------- double-float refinement
// Closest hits get t, u, v recomputed in double-float arithmetic (hi + lo floats, about
// 48 significant bits) on the float32 pipes, FP64 running at a small fraction of their
// rate on this GPU. Addition and multiplication are the accurate double-word algorithms
// of Joldes, Muller and Popescu ("Tight and Rigorous Error Bounds for Basic Building
// Blocks of Double-Word Arithmetic", ACM TOMS 2017: relative errors of a few u^2), built
// on Dekker's and Knuth's error-free transformations; division and square root take one
// Newton correction of the float32 quotient or root.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ffOf(float a) { return FF{a, 0.f}; }
__device__ __forceinline__ FF ffFast(float a, float b) {  // |a| >= |b| (or a = 0)
    const float s = __fadd_rn(a, b);
    return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ffAdd(FF a, FF b) {
    const float2 s = twoSum(a.hi, b.hi), t = twoSum(a.lo, b.lo);
    const FF v = ffFast(s.x, __fadd_rn(s.y, t.x));
    return ffFast(v.hi, __fadd_rn(t.y, v.lo));
}
__device__ __forceinline__ FF ffSub(FF a, FF b) { return ffAdd(a, FF{-b.hi, -b.lo}); }
__device__ __forceinline__ FF ffMul(FF a, FF b) {
    const float2 c = twoProd(a.hi, b.hi);
    const float tl = fmaf(a.lo, b.hi, __fmul_rn(a.hi, b.lo));
    return ffFast(c.x, __fadd_rn(c.y, tl));
}
__device__ __forceinline__ FF ffDiv(FF a, FF b) {
    const float q = __fdiv_rn(a.hi, b.hi);
    const FF r = ffSub(a, ffMul(b, ffOf(q)));  // the remainder of the float32 quotient
    return ffFast(q, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ FF ffSqrt(FF a) {
    if (!(a.hi > 0.f)) return FF{0.f, 0.f};
    const float r = sqrtf(a.hi);
    const FF e = ffSub(a, ffMul(ffOf(r), ffOf(r)));
    return ffFast(r, __fdiv_rn(e.hi, __fmul_rn(2.f, r)));
}
__device__ __forceinline__ float ffRound(FF a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ FF ffDot(const FF a[3], const FF b[3]) {
    return ffAdd(ffAdd(ffMul(a[0], b[0]), ffMul(a[1], b[1])), ffMul(a[2], b[2]));
}
__device__ __forceinline__ void ffCross(const FF a[3], const FF b[3], FF c[3]) {
    c[0] = ffSub(ffMul(a[1], b[2]), ffMul(a[2], b[1]));
    c[1] = ffSub(ffMul(a[2], b[0]), ffMul(a[0], b[2]));
    c[2] = ffSub(ffMul(a[0], b[1]), ffMul(a[1], b[0]));
}

// The ray at the hit's level in double-float: the world ray itself, or its image under
// the instance's inverse frame held as float32 rows (hi) plus low parts (lo), hi + lo
// being the FP64 frame to 2^-48.
__device__ __forceinline__ void rayFF(const float4* hi, const float4* lo, float3 wo, float3 wd, FF o[3], FF d[3]) {
    if (!hi) {
        o[0] = ffOf(wo.x), o[1] = ffOf(wo.y), o[2] = ffOf(wo.z);
        d[0] = ffOf(wd.x), d[1] = ffOf(wd.y), d[2] = ffOf(wd.z);
        return;
    }
    const float w[3] = {wo.x, wo.y, wo.z}, v[3] = {wd.x, wd.y, wd.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 H = __ldg(hi + k), L = __ldg(lo + k);
        const FF g[3] = {FF{H.x, L.x}, FF{H.y, L.y}, FF{H.z, L.z}};
        FF ok = FF{H.w, L.w}, dk = FF{0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            ok = ffAdd(ok, ffMul(g[j], ffOf(w[j])));
            dk = ffAdd(dk, ffMul(g[j], ffOf(v[j])));
        }
        o[k] = ok, d[k] = dk;
    }
}

// The closest hit's (t, u, v, 1) recomputed in double-float (Moller-Trumbore on the
// level's ray, or the sphere quadratic's root in [tmin, tmax]); w = 0 when it cannot
// be evaluated (the float32 values then stand).
static __device__ __noinline__ float4 refineFF(const float4* hi, const float4* lo, float3 wo, float3 wd,
                                              const float4* rec, bool sphere, float tmin, float tmax) {
    FF o[3], d[3];
    rayFF(hi, lo, wo, wd, o, d);
    if (sphere) {
        const float4 sp = __ldg(rec);
        const FF f[3] = {ffAdd(o[0], ffOf(-sp.x)), ffAdd(o[1], ffOf(-sp.y)), ffAdd(o[2], ffOf(-sp.z))};
        const FF a = ffDot(d, d), b = ffDot(f, d);
        const FF c = ffSub(ffDot(f, f), ffMul(ffOf(sp.w), ffOf(sp.w)));
        const FF disc = ffSub(ffMul(b, b), ffMul(a, c));
        if (disc.hi < 0.f || a.hi == 0.f) return make_float4(0.f, 0.f, 0.f, 0.f);
        const FF q = ffSqrt(disc), nb = FF{-b.hi, -b.lo};
        const float t0 = ffRound(ffDiv(ffSub(nb, q), a)), t1 = ffRound(ffDiv(ffAdd(nb, q), a));
        if (t0 >= tmin && t0 <= tmax) return make_float4(t0, 0.f, 0.f, 1.f);
        if (t1 >= tmin && t1 <= tmax) return make_float4(t1, 0.f, 0.f, 1.f);
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 A = __ldg(rec), B = __ldg(rec + 1), C = __ldg(rec + 2);
    const float2 x1 = twoSum(B.x, -A.x), y1 = twoSum(B.y, -A.y), z1 = twoSum(B.z, -A.z);
    const float2 x2 = twoSum(C.x, -A.x), y2 = twoSum(C.y, -A.y), z2 = twoSum(C.z, -A.z);
    const FF e1[3] = {FF{x1.x, x1.y}, FF{y1.x, y1.y}, FF{z1.x, z1.y}};
    const FF e2[3] = {FF{x2.x, x2.y}, FF{y2.x, y2.y}, FF{z2.x, z2.y}};
    FF P[3], Q[3];
    ffCross(d, e2, P);
    const FF det = ffDot(e1, P);
    if (det.hi == 0.f) return make_float4(0.f, 0.f, 0.f, 0.f);
    const FF T[3] = {ffAdd(o[0], ffOf(-A.x)), ffAdd(o[1], ffOf(-A.y)), ffAdd(o[2], ffOf(-A.z))};
    ffCross(T, e1, Q);
    return make_float4(ffRound(ffDiv(ffDot(e2, Q), det)), ffRound(ffDiv(ffDot(T, P), det)),
                       ffRound(ffDiv(ffDot(d, Q), det)), 1.f);
}

// Enter an instance. The object-space origin is placed where the world ray enters the
// instance's world box (world parameter tOff) and computed to near-FP64 accuracy (see
// instanceOriginFF), so that it is small and correctly rounded: float32 differences to
// nearby vertices then lose little. The direction is transformed in float32 with a
// bound on its error (matrix entries rounded from FP64 plus three rounded FMAs per
// component). Boxes are widened by the worst position error over the instance's
// parameter range.
__device__ __forceinline__ void instanceLevel(Level& L, const InstanceRecord* R, const float4* frames32, float3 wo,
                                              float3 wd, float3 wid, float tmin, float lim) {
    const float4 m[3] = {R->inv[0], R->inv[1], R->inv[2]};
    const float4 blo = R->worldLo, bhi = R->worldHi;
    // entry and exit parameters of the world box (exact world ray, conservative)
    const bool px = wid.x >= 0.f, py = wid.y >= 0.f, pz = wid.z >= 0.f;
    const float nx = ((px ? blo.x : bhi.x) - wo.x) * wid.x, fx = ((px ? bhi.x : blo.x) - wo.x) * wid.x;
    const float ny = ((py ? blo.y : bhi.y) - wo.y) * wid.y, fy = ((py ? bhi.y : blo.y) - wo.y) * wid.y;
    const float nz = ((pz ? blo.z : bhi.z) - wo.z) * wid.z, fz = ((pz ? bhi.z : blo.z) - wo.z) * wid.z;
    const float tentry = fmaxf(fmaxf(nx, ny), fmaxf(nz, tmin));
    const float texit = fminf(fminf(fx, fy), fminf(fz, lim)) * kFarScale;
    const float te = (tentry < texit && tentry < INFINITY) ? tentry : tmin;  // any finite shift is exact enough
    const float3 og = instanceOriginFF(R->inv, frames32 + kFrameRows * (size_t)R->instanceID + 3, wo, wd, te);
    const float o[3] = {og.x, og.y, og.z};
    float d[3], sd = 0.f, so = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d[k] = fmaf(m[k].x, wd.x, fmaf(m[k].y, wd.y, m[k].z * wd.z));
        sd = fmaxf(sd, fabsf(m[k].x * wd.x) + fabsf(m[k].y * wd.y) + fabsf(m[k].z * wd.z));
        so = fmaxf(so, fabsf(o[k]));
    }
    L.o = make_float3(o[0], o[1], o[2]);
    L.d = make_float3(d[0], d[1], d[2]);
    L.id = make_float3(__frcp_rn(d[0]), __frcp_rn(d[1]), __frcp_rn(d[2]));
    L.dl1 = norm1(L.d);
    L.tOff = te;
    // final rounding (u) plus the float-float evaluation's own error (tens of u^2
    // relative to the largest term, which is at most about 2^10 times |o| here)
    L.dO = 1.01f * kEps * so + 64.f * kEps * kEps * (so + fabsf(m[0].w) + fabsf(m[1].w) + fabsf(m[2].w) +
                                                  fabsf(te) * L.dl1 + norm1(wo) * 4.f) + 1e-30f;
    L.dD = 6.f * kEps * sd;
    const float span = fmaxf(fabsf(texit - te), fabsf(tmin - te)) * (1.f + 4.f * kEps);
    const float slack = L.dO + span * L.dD + 2.f * kEps * so;
    const float3 sg = make_float3(copysignf(slack, L.id.x), copysignf(slack, L.id.y), copysignf(slack, L.id.z));
    L.on = L.o + sg;
    L.of = L.o - sg;
}

struct Stack {
    uint32_t* sh;
    uint32_t* gl;
    uint32_t shDepth, glDepth, stride, sp;
    __device__ __forceinline__ bool push(uint32_t x) {
        if (sp < shDepth) {
            sh[sp * blockDim.x] = x;
        } else if (sp < shDepth + glDepth) {
            gl[(size_t)(sp - shDepth) * stride] = x;
        } else {
            return false;
        }
        ++sp;
        return true;
    }
    __device__ __forceinline__ uint32_t pop() {
        --sp;
        return sp < shDepth ? sh[sp * blockDim.x] : gl[(size_t)(sp - shDepth) * stride];
    }
    __device__ __forceinline__ uint32_t top() const {
        const uint32_t i = sp - 1;
        return i < shDepth ? sh[i * blockDim.x] : gl[(size_t)(i - shDepth) * stride];
    }
};

// Per-ray work counts (only with COUNT): nodes, triangles, customs, instances, FP64 tests.
struct Visits {
    uint32_t nodes = 0, tris = 0, customs = 0, insts = 0, fp64 = 0;
};

__device__ __forceinline__ void flushVisits(unsigned long long* stats, const Visits& v) {
    atomicAdd(&stats[0], 1ull);
    atomicAdd(&stats[1], (unsigned long long)v.nodes);
    atomicAdd(&stats[2], (unsigned long long)v.tris);
    atomicAdd(&stats[3], (unsigned long long)v.customs);
    atomicAdd(&stats[4], (unsigned long long)v.insts);
    atomicAdd(&stats[5], (unsigned long long)v.fp64);
}

// Traversal state of one ray, kept in registers between steps.
struct RayState {
    float3 wo, wd, wid;  // world ray and its reciprocal direction
    float tmin, tmax;
    Level L;             // ray at the current level
    const float4* nodes;
    const void* leaves;
    Hit best;
    uint32_t primType, geomType, instId;
    uint32_t steps, next;
    float lo, hi;  // [tmin, limit] on the current level (limit = tmax, or the best t so far)
    bool inBlas, found;
    uint32_t fmt;  // the current level's node format (TraceTarget::fmt)
};

// The slab test of the current node in the current level's node format, over the W =
// slotsOf(FM) entries of tn and c; a 4-wide level in a W = 8 walk fills the first four
// and marks the rest empty.
template <int FM>
__device__ __forceinline__ uint32_t slabNode(const RayState& s, float* tn, uint32_t* c) {
    if constexpr (FM == kFmPlain) {
        return slab4(s.nodes, s.next, s.L, s.lo, s.hi, tn, c);
    } else if constexpr (FM == kFmWide8) {
        return slab8(s.nodes, s.next, s.L, s.lo, s.hi, tn, c);
    } else if constexpr (FM == kFmQuant) {
        return s.fmt == 1u ? slab4q(s.nodes, s.next, s.L, s.lo, s.hi, tn, c)
                           : slab4(s.nodes, s.next, s.L, s.lo, s.hi, tn, c);
    } else {
        if (s.fmt == 2u) return slab8(s.nodes, s.next, s.L, s.lo, s.hi, tn, c);
#pragma unroll
        for (int j = 4; j < 8; ++j) c[j] = kInvalid, tn[j] = INFINITY;
        return s.fmt == 1u ? slab4q(s.nodes, s.next, s.L, s.lo, s.hi, tn, c)
                           : slab4(s.nodes, s.next, s.L, s.lo, s.hi, tn, c);
    }
}

template <bool SCENE>
__device__ __forceinline__ void beginRay(const TraceParams& P, Stack& st, RayState& s, float3 wo, float3 wd,
                                         float tmin, float tmax) {
    s.best = Hit{kInvalid, kInvalid, INFINITY, 0.f, 0.f};
    s.wo = wo;
    s.wd = wd;
    s.tmin = tmin;
    s.tmax = tmax;
    exactLevel(s.L, wo, wd);
    s.wid = s.L.id;
    s.nodes = P.target.nodes;
    s.fmt = P.target.fmt;
    s.leaves = P.target.leaves;
    s.primType = P.target.primType;
    s.geomType = P.target.geomType;
    s.instId = 0;
    s.inBlas = !SCENE;
    s.found = false;
    s.steps = 0;
    s.next = P.target.empty ? kNone : 0u;
    s.lo = tmin;  // the world level: local = world parameters
    s.hi = tmax;
    st.sp = 0;
}

// Moves the ray into instance R (a top-level leaf): the ray in R's object space, R's
// bottom level as the current level, and a marker on the stack that brings the ray
// back to the top level when R's traversal is done. False when nothing was entered.
template <bool ANY, bool COUNT>
__device__ __forceinline__ bool enterInstance(const TraceParams& P, Stack& st, RayState& s, const InstanceRecord* R,
                                              Visits* vis) {
    const uint32_t bits = R->typeBits;
    if ((bits & kInstEmpty) || !(R->mask & P.rayMask)) return false;
    if (!st.push(kSentinel)) {
        latchError(P.error, GRT_ERROR_STACK_OVERFLOW);
        return false;
    }
    if (COUNT) ++vis->insts;
    const float lim = (ANY || !s.found) ? s.tmax : s.best.t;
    instanceLevel(s.L, R, P.fwd32, s.wo, s.wd, s.wid, s.tmin, lim);
    s.lo = localLo(s.L, s.tmin);
    s.hi = localHi(s.L, lim);
    s.nodes = R->nodes;
    s.fmt = (bits & kInstQuant) ? 1u : (bits & kInstWide8) ? 2u : 0u;
    s.leaves = R->leaves;
    s.primType = instPrimType(bits);
    s.geomType = instGeomType(bits);
    s.instId = R->instanceID;
    s.inBlas = true;
    s.next = 0;
    return true;
}

// Tests leaf k of the current level against the ray (closest hit: only nearer than
// the best so far). Returns true when it is a hit; s.best then holds it.
// The ray of level L as a grtRay over world parameters [a, b]: origin at world
// parameter L.tOff, so that t on it is the world parameter minus L.tOff.
__device__ __forceinline__ grtRay levelRay(const Level& L, float a, float b) {
    grtRay r;
    r.origin[0] = L.o.x, r.origin[1] = L.o.y, r.origin[2] = L.o.z;
    r.direction[0] = L.d.x, r.direction[1] = L.d.y, r.direction[2] = L.d.z;
    r.minT = a - L.tOff;
    r.maxT = b - L.tOff;
    return r;
}

template <bool ANY, bool SCENE, bool COUNT, class U = NoUser>
__device__ __forceinline__ bool testLeaf(const TraceParams& P, RayState& s, uint32_t k, Visits* vis,
                                         const U* user = nullptr, void* payload = nullptr) {
    const bool strict = s.found && !ANY;
    const float cur = (ANY || !s.found) ? s.tmax : s.best.t;
    float t = 0.f, u = 0.f, v = 0.f;
    uint32_t prim;
    int res = 0;
    const float4* rec;
    bool sphere = false;
    if (s.primType == GRT_PRIMITIVE_TRIANGLE_MESH) {
        rec = reinterpret_cast<const float4*>(s.leaves) + 3 * (size_t)k;
        const float4 a = __ldg(rec), b = __ldg(rec + 1), e = __ldg(rec + 2);
        prim = __float_as_uint(a.w);
        res = triangleTest(s.L, f3(a), f3(b), f3(e), b.w, e.w, s.tmin, cur, strict, t, u, v);
        if (COUNT) ++vis->tris;
        if (res == 2) {
            if (COUNT) ++vis->fp64;
            const float4 r = decide64(P.inv64, SCENE, s.instId, s.wo, s.wd, rec, false, s.tmin, cur, strict);
            res = r.w != 0.f ? 1 : 0;
            t = r.x, u = r.y, v = r.z;
        }
    } else {
        prim = __ldg(reinterpret_cast<const uint32_t*>(s.leaves) + k);
        rec = nullptr;
        if (P.table && s.geomType < P.numGeomTypes) {
            const FuncEntry fe = P.table[(size_t)P.rayType * P.numGeomTypes + s.geomType];
            if (fe.func == GRT_INTERSECT_SPHERE) {
                rec = reinterpret_cast<const float4*>(fe.data) + prim;
                sphere = true;
                const float4 sp = __ldg(rec);
                res = sphereTest(s.L, sp, s.tmin, cur, strict, t);
                if (COUNT) ++vis->customs;
                if (res == 2) {
                    if (COUNT) ++vis->fp64;
                    const float4 r =
                        decide64(P.inv64, SCENE, s.instId, s.wo, s.wd, rec, true, s.tmin, cur, strict);
                    res = r.w != 0.f ? 1 : 0;
                    t = r.x, u = r.y, v = r.z;
                }
            } else if constexpr (kHasUser<U>) {
                if (fe.func >= GRT_INTERSECT_USER) {  // user code (Sec. 7.4): its t is on the level's ray
                    if (COUNT) ++vis->customs;
                    grtHit h;
                    h.instanceID = s.instId, h.primID = prim, h.t = INFINITY, h.u = 0.f, h.v = 0.f;
                    if (user->intersect(fe.func, levelRay(s.L, s.tmin, cur), fe.data, payload, h)) {
                        const float tw = h.t + s.L.tOff;
                        if (tw >= s.tmin && (strict ? tw < cur : tw <= cur)) res = 1, t = tw, u = h.u, v = h.v;
                    }
                }
            }
        }
    }
    if (res == 1 && P.table && s.geomType < P.numGeomTypes) {  // intersection filter (Sec. 7.6)
        const FuncEntry* fe = P.table + (size_t)P.rayType * P.numGeomTypes + s.geomType;
        if (fe->filter == GRT_FILTER_PRIMITIVE_MASK) {
            const uint32_t* bits = static_cast<const uint32_t*>(fe->filterData);
            if (!((__ldg(bits + (prim >> 5)) >> (prim & 31u)) & 1u)) res = 0;
        } else if constexpr (kHasUser<U>) {
            if (fe->filter >= GRT_FILTER_USER) {
                grtHit h;
                h.instanceID = s.instId, h.primID = prim, h.t = t - s.L.tOff, h.u = u, h.v = v;
                if (!user->filter(fe->filter, levelRay(s.L, s.tmin, cur), fe->filterData, payload, h)) res = 0;
            }
        }
    }
    if (res == 1) {
        s.best = Hit{s.instId, prim, t, u, v};
        s.found = true;
        if (!ANY) s.hi = localHi(s.L, t);
        return true;
    }
    return false;
}

__device__ __forceinline__ void sort2(uint32_t& a, uint32_t& b) {
    const uint32_t x = min(a, b);
    b = max(a, b);
    a = x;
}

// The slots in mask m go on: the nearest (smallest entry distance) becomes s.next and
// the others are pushed, farthest first, so that they come off the stack near to far.
// Two slots take one comparison; three or four go through a sorting network on keys
// made of the entry distance as an ordered integer with the slot in its two low bits.
__device__ __forceinline__ void orderChildren(const TraceParams& P, Stack& st, RayState& s, uint32_t m,
                                              const float tn[4], const uint32_t c[4]) {
    if (m == 0) return;
    if ((m & (m - 1u)) == 0) {
        s.next = pick4(c, (uint32_t)__ffs(m) - 1u);
        return;
    }
    if (__popc(m) == 2) {  // the most frequent case after a single hit: one comparison
        const uint32_t a = (uint32_t)__ffs(m) - 1u, b = 31u - (uint32_t)__clz(m);
        const float ta = a == 0 ? tn[0] : a == 1 ? tn[1] : tn[2];
        const float tb = b == 1 ? tn[1] : b == 2 ? tn[2] : tn[3];
        const uint32_t ca = pick4(c, a), cb = pick4(c, b);
        const bool swap = tb < ta;
        if (!st.push(swap ? ca : cb)) latchError(P.error, GRT_ERROR_STACK_OVERFLOW);
        s.next = swap ? cb : ca;
        return;
    }
    uint32_t k[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) k[j] = ((m >> j) & 1u) ? ((floatToOrdered(tn[j]) & ~3u) | (uint32_t)j) : kInvalid;
    sort2(k[0], k[1]);
    sort2(k[2], k[3]);
    sort2(k[0], k[2]);
    sort2(k[1], k[3]);
    sort2(k[1], k[2]);
    bool ok = true;
    if (k[3] != kInvalid) ok &= st.push(pick4(c, k[3] & 3u));
    if (k[2] != kInvalid) ok &= st.push(pick4(c, k[2] & 3u));
    ok &= st.push(pick4(c, k[1] & 3u));
    if (!ok) latchError(P.error, GRT_ERROR_STACK_OVERFLOW);
    s.next = pick4(c, k[0] & 3u);
}

template <class T>
__device__ __forceinline__ T pick8(const T v[8], uint32_t j) {
    T r = v[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) r = j == (uint32_t)i ? v[i] : r;
    return r;
}

// orderChildren for an 8-wide visit: one or two slots as there; three or more through
// Batcher's odd-even merge network for eight keys (19 comparators) on (entry distance,
// slot) keys, the slot in the three low bits.
__device__ __forceinline__ void orderChildren8(const TraceParams& P, Stack& st, RayState& s, uint32_t m,
                                               const float tn[8], const uint32_t c[8]) {
    if (m == 0) return;
    if ((m & (m - 1u)) == 0) {
        s.next = pick8(c, (uint32_t)__ffs(m) - 1u);
        return;
    }
    if (__popc(m) == 2) {
        const uint32_t a = (uint32_t)__ffs(m) - 1u, b = 31u - (uint32_t)__clz(m);
        const uint32_t ca = pick8(c, a), cb = pick8(c, b);
        const bool swap = pick8(tn, b) < pick8(tn, a);
        if (!st.push(swap ? ca : cb)) latchError(P.error, GRT_ERROR_STACK_OVERFLOW);
        s.next = swap ? cb : ca;
        return;
    }
    uint32_t k[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) k[j] = ((m >> j) & 1u) ? ((floatToOrdered(tn[j]) & ~7u) | (uint32_t)j) : kInvalid;
    sort2(k[0], k[1]), sort2(k[2], k[3]), sort2(k[4], k[5]), sort2(k[6], k[7]);
    sort2(k[0], k[2]), sort2(k[1], k[3]), sort2(k[4], k[6]), sort2(k[5], k[7]);
    sort2(k[1], k[2]), sort2(k[5], k[6]);
    sort2(k[0], k[4]), sort2(k[1], k[5]), sort2(k[2], k[6]), sort2(k[3], k[7]);
    sort2(k[2], k[4]), sort2(k[3], k[5]);
    sort2(k[1], k[2]), sort2(k[3], k[4]), sort2(k[5], k[6]);
    bool ok = true;
#pragma unroll
    for (int j = 7; j >= 1; --j)
        if (k[j] != kInvalid) ok &= st.push(pick8(c, k[j] & 7u));
    if (!ok) latchError(P.error, GRT_ERROR_STACK_OVERFLOW);
    s.next = pick8(c, k[0] & 7u);
}

template <int W>
__device__ __forceinline__ void orderSlots(const TraceParams& P, Stack& st, RayState& s, uint32_t m, const float* tn,
                                           const uint32_t* c) {
    if constexpr (W == 8)
        orderChildren8(P, st, s, m, tn, c);
    else
        orderChildren(P, st, s, m, tn, c);
}

// An any-hit step takes the hit children in slot order, without sorting them by entry
// distance: any hit ends the walk, and the sort cost more than its early exits saved
// (1M spheres any hit 2.80 -> 2.72 ms, terrain AO 0.726 -> 0.723 ms, dense-view AO 6.75
// -> 6.67 ms). Closest hits keep the near-first order.
template <int W, bool ANY>
__device__ __forceinline__ void orderSlotsQ(const TraceParams& P, Stack& st, RayState& s, uint32_t m, const float* tn,
                                            const uint32_t* c) {
    if constexpr (ANY) {
        if (m == 0) return;
        const uint32_t first = (uint32_t)__ffs(m) - 1u;
        m &= m - 1u;
        bool ok = true;
        while (m) {
            const uint32_t j = 31u - (uint32_t)__clz(m);
            m &= ~(1u << j);
            if constexpr (W == 8)
                ok &= st.push(pick8(c, j));
            else
                ok &= st.push(pick4(c, j));
        }
        if (!ok) latchError(P.error, GRT_ERROR_STACK_OVERFLOW);
        if constexpr (W == 8)
            s.next = pick8(c, first);
        else
            s.next = pick4(c, first);
    } else {
        orderSlots<W>(P, st, s, m, tn, c);
    }
}

// One traversal step: a node visit (with its leaf tests), an instance entry or an
// instance exit. Returns true once the ray is finished (s.best is then final).
template <bool ANY, bool SCENE, bool COUNT, class U = NoUser, int FM = kFmMixed>
__device__ __forceinline__ bool stepRay(const TraceParams& P, Stack& st, RayState& s, Visits* vis,
                                        const U* user = nullptr, void* payload = nullptr) {
    if (s.next == kNone) {
        if (st.sp == 0) return true;  // closest hits are refined afterwards (refineKernel)
        s.next = st.pop();
        if (SCENE && s.next == kSentinel) {  // back to the top level
            exactLevel(s.L, s.wo, s.wd);
            s.lo = s.tmin;
            s.hi = (ANY || !s.found) ? s.tmax : s.best.t;
            s.nodes = P.target.nodes;
            s.fmt = P.target.fmt;
            s.inBlas = false;
            s.next = kNone;
            return false;
        }
    }
    if (SCENE && !s.inBlas && (s.next & kLeafBit)) {  // enter an instance
        const uint32_t leaf = s.next & ~kLeafBit;
        s.next = kNone;
        enterInstance<ANY, COUNT>(P, st, s, reinterpret_cast<const InstanceRecord*>(P.target.leaves) + leaf, vis);
        return false;
    }
    if (++s.steps > P.maxSteps) {
        latchError(P.error, GRT_ERROR_STEP_LIMIT);
        return true;
    }
    if (COUNT) ++vis->nodes;
    constexpr int W = slotsOf(FM);
    float tn[W];
    uint32_t c[W];
    uint32_t m = slabNode<FM>(s, tn, c);
    s.next = kNone;
    if (s.inBlas) {  // one copy of the leaf test (a large inlined body), over the hit leaf slots
        uint32_t lm = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) lm |= (c[j] & kLeafBit) ? (1u << j) : 0u;
        lm &= m;
        m &= ~lm;
        while (lm) {
            const uint32_t j = (uint32_t)__ffs(lm) - 1u;
            lm &= lm - 1u;
            uint32_t cj;
            if constexpr (W == 8)
                cj = pick8(c, j);
            else
                cj = pick4(c, j);
            if (testLeaf<ANY, SCENE, COUNT, U>(P, s, cj & ~kLeafBit, vis, user, payload) && ANY) return true;
        }
    }
    orderSlotsQ<W, ANY>(P, st, s, m, tn, c);
    return false;
}

// One step of an all-hits walk (Sec. 7.5: every intersection, found by asking the
// any-hit traversal for its next hit until it is done): a node visit that tests every
// leaf it reaches against the whole range [tmin, tmax] and appends each hit to `found`
// (at most W = slotsOf(FM) per visit), or an instance entry or exit. Returns the number of hits
// appended, or -1 once the walk is over. Each primitive of each instance sits in one
// leaf, so each (instance, primitive) is reported at most once; an instance of a geometry
// with split triangles (several leaves per triangle) is skipped and latches
// GRT_ERROR_INVALID_PARAMETER.
template <bool SCENE, class U = NoUser, int FM = kFmMixed>
__device__ __forceinline__ int stepAll(const TraceParams& P, Stack& st, RayState& s, Hit* found,
                                       const U* user = nullptr, void* payload = nullptr) {
    if (s.next == kNone) {
        if (st.sp == 0) return -1;
        s.next = st.pop();
        if (SCENE && s.next == kSentinel) {  // back to the top level
            exactLevel(s.L, s.wo, s.wd);
            s.lo = s.tmin;
            s.hi = s.tmax;
            s.nodes = P.target.nodes;
            s.fmt = P.target.fmt;
            s.inBlas = false;
            s.next = kNone;
            return 0;
        }
    }
    if (SCENE && !s.inBlas && (s.next & kLeafBit)) {  // enter an instance
        const uint32_t leaf = s.next & ~kLeafBit;
        s.next = kNone;
        s.found = false;
        const InstanceRecord* R = reinterpret_cast<const InstanceRecord*>(P.target.leaves) + leaf;
        if (R->typeBits & kInstSplit)
            latchError(P.error, GRT_ERROR_INVALID_PARAMETER);
        else
            enterInstance<true, false>(P, st, s, R, nullptr);
        return 0;
    }
    if (++s.steps > P.maxSteps) {
        latchError(P.error, GRT_ERROR_STEP_LIMIT);
        return -1;
    }
    constexpr int W = slotsOf(FM);
    float tn[W];
    uint32_t c[W];
    uint32_t m = slabNode<FM>(s, tn, c);
    s.next = kNone;
    int added = 0;
    if (s.inBlas) {
        uint32_t lm = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) lm |= (c[j] & kLeafBit) ? (1u << j) : 0u;
        lm &= m;
        m &= ~lm;
        while (lm) {  // one copy of the leaf test, over the hit leaf slots
            const uint32_t j = (uint32_t)__ffs(lm) - 1u;
            lm &= lm - 1u;
            uint32_t cj;
            if constexpr (W == 8)
                cj = pick8(c, j);
            else
                cj = pick4(c, j);
            if (testLeaf<true, SCENE, false, U>(P, s, cj & ~kLeafBit, nullptr, user, payload)) found[added++] = s.best;
        }
    }
    orderSlots<W>(P, st, s, m, tn, c);
    return added;
}

// One ray through the target, all steps in a row. Returns the hit (prim == kInvalid
// on a miss).
template <bool ANY, bool SCENE, bool COUNT = false, class U = NoUser>
__device__ Hit traceRay(const TraceParams& P, Stack& st, float3 wo, float3 wd, float tmin, float tmax,
                        Visits* vis = nullptr, const U* user = nullptr, void* payload = nullptr) {
    RayState s;
    beginRay<SCENE>(P, st, s, wo, wd, tmin, tmax);
    while (!stepRay<ANY, SCENE, COUNT, U>(P, st, s, vis, user, payload)) {
    }
    return s.best;
}

__device__ __forceinline__ void storeHit(uint32_t* hits, uint32_t r, const Hit& h) {
    uint32_t* p = hits + 5 * (size_t)r;
    p[0] = h.inst;
    p[1] = h.prim;
    p[2] = __float_as_uint(h.t);
    p[3] = __float_as_uint(h.u);
    p[4] = __float_as_uint(h.v);
}

// ---------------------------------------------------------------- ambient occlusion rays (Sec. 4)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// splitmix64 value at counter (pixel << 32 | sample << 1 | dim) of stream `seed`, top 24 bits.
__device__ __forceinline__ float sampleXi(uint64_t seed, uint64_t pixel, uint32_t sample, uint32_t dim) {
    const uint64_t c = (pixel << 32) | ((uint64_t)sample << 1) | dim;
    const uint64_t h = mix64(seed + (c + 1ull) * 0x9E3779B97F4A7C15ull);
    return (float)(uint32_t)(h >> 40) * 5.9604644775390625e-8f;
}

struct AoFrame {
    float3 org, n, tg, bt;
};

// World hit point, face normal turned toward the viewer, and the tangent frame of
// the triangle a primary ray hit.
__device__ __forceinline__ bool aoFrame(const InstanceRecord* sceneLeaves, const uint32_t* scenePrimToLeaf,
                                        const float4* fwd32, const float4* ray, const uint32_t* hit, AoFrame& F) {
    const uint32_t inst = hit[0], prim = hit[1];
    if (prim == kInvalid) return false;
    const InstanceRecord* R = sceneLeaves + scenePrimToLeaf[inst];
    if (instPrimType(R->typeBits) != GRT_PRIMITIVE_TRIANGLE_MESH) return false;
    const BvhHeader* g = R->geometry;
    const float4* rec = reinterpret_cast<const float4*>(g->leaves) + 3 * (size_t)g->primToLeaf[prim];
    const float4* fr = fwd32 + kFrameRows * (size_t)inst;
    const float4 m0 = fr[0], m1 = fr[1], m2 = fr[2];
    // world edges = linear part of the frame applied to object-space edges (no
    // cancellation against the translation)
    const float3 v0 = f3(rec[0]), a1 = f3(rec[1]) - v0, a2 = f3(rec[2]) - v0;
    const float3 e1 = make_float3(m0.x * a1.x + m0.y * a1.y + m0.z * a1.z, m1.x * a1.x + m1.y * a1.y + m1.z * a1.z,
                                  m2.x * a1.x + m2.y * a1.y + m2.z * a1.z);
    const float3 e2 = make_float3(m0.x * a2.x + m0.y * a2.y + m0.z * a2.z, m1.x * a2.x + m1.y * a2.y + m1.z * a2.z,
                                  m2.x * a2.x + m2.y * a2.y + m2.z * a2.z);
    const float4 a = ray[0], b = ray[1];
    const float3 o = f3(a), d = f3(b);
    float3 n = normalize3(cross3(e1, e2));
    if (dot3(n, d) > 0.0f) n = n * -1.0f;
    F.n = n;
    F.tg = normalize3(e1);
    F.bt = cross3(n, F.tg);
    const float t = __uint_as_float(hit[2]);
    F.org = (o + d * t) + n * 1e-4f;
    return true;
}

__device__ __forceinline__ float3 aoDirection(const AoFrame& F, uint64_t seed, uint64_t pixel, uint32_t s) {
    const float xi0 = sampleXi(seed, pixel, s, 0), xi1 = sampleXi(seed, pixel, s, 1);
    float sn, cs;
    sincospif(2.0f * xi0, &sn, &cs);
    const float r = sqrtf(xi1);
    // y = sqrt(1 - r^2) = sqrt(1 - xi1): xi1 is a multiple of 2^-24 in [0, 1), so 1 - xi1
    // is exact in float32, where 1 - r*r would cancel for grazing samples (xi1 near 1)
    const float x = cs * r, z = sn * r, y = sqrtf(1.0f - xi1);
    return F.tg * x + F.bt * z + F.n * y;
}

// Refill loop with one traversal step per lane per iteration (node visits test their
// leaves at once). Used for any-hit queries on a single geometry (shadow rays), which
// stop at their first hit and so gain nothing from queueing leaves.
template <bool ANY, bool SCENE, bool COUNT, int FM = kFmMixed, class Src>
__device__ __forceinline__ void refillLoopPerRay(const TraceParams& P, Stack& st, Src& src) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t ltMask = (1u << lane) - 1u;
    const unsigned long long total = src.count();
    RayState s;
    Visits v;
    uint32_t item = kNone;
    bool exhausted = false;
    for (;;) {
        uint32_t live = __ballot_sync(0xffffffffu, item != kNone);
        while (!exhausted && (uint32_t)__popc(live) <= P.refillBelow) {
            const uint32_t idle = ~live;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(P.counter, (unsigned long long)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base + __popc(idle) >= total) exhausted = true;
            if (item == kNone) {
                const unsigned long long mine = base + __popc(idle & ltMask);
                if (mine < total && src.begin((uint32_t)mine, P, st, s)) {
                    item = (uint32_t)mine;
                    if (COUNT) v = Visits{};
                }
            }
            live = __ballot_sync(0xffffffffu, item != kNone);
        }
        if (live == 0) break;
        if (item != kNone && stepRay<ANY, SCENE, COUNT, NoUser, FM>(P, st, s, &v)) {
            src.finish(item, s);
            if (COUNT) flushVisits(P.stats, v);
            item = kNone;
        }
    }
}

// ---------------------------------------------------------------- phased warp traversal
// What a lane does next. NODE: visit s.next; ENTER: enter the instance at top-level
// leaf s.next; FLUSH: test its pending leaves before anything else (its queue is too
// full for another node visit, or its ray is about to leave the current instance or
// to finish); DONE: the ray is finished.
enum : uint32_t { kStNode = 0, kStEnter = 1, kStFlush = 2, kStDone = 3 };

// Leaves of the current bottom level whose boxes the ray hit, waiting to be tested:
// at most pendingCap(W), in shared memory after the lane's stack slice (entry i at
// buf[i * blockDim.x]). Kernels running refillLoop reserve traceSmemWords(depth, W)
// words of shared memory per thread.
struct Pending {
    uint32_t* buf;
    uint32_t n;
    __device__ __forceinline__ void add(uint32_t k) {
        buf[n * blockDim.x] = k;
        ++n;
    }
    __device__ __forceinline__ uint32_t at(uint32_t i) const { return buf[i * blockDim.x]; }
};

// Node visit that queues hit leaf children instead of testing them (inner children
// and top-level leaves go on as in stepRay). Requires q.n <= pendingCap(W) - W.
template <bool ANY, bool SCENE, bool COUNT, int FM = kFmMixed>
__device__ __forceinline__ void visitNode(const TraceParams& P, Stack& st, RayState& s, Pending& q, Visits* vis) {
    if (++s.steps > P.maxSteps) {
        latchError(P.error, GRT_ERROR_STEP_LIMIT);
        s.next = kNone;
        st.sp = 0;
        q.n = 0;
        return;
    }
    if (COUNT) ++vis->nodes;
    constexpr int W = slotsOf(FM);
    float tn[W];
    uint32_t c[W];
    uint32_t m = slabNode<FM>(s, tn, c);
    s.next = kNone;
    if (s.inBlas) {
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (((m >> j) & 1u) && (c[j] & kLeafBit)) q.add(c[j] & ~kLeafBit), m &= ~(1u << j);
    }
    orderSlots<W>(P, st, s, m, tn, c);
}

// The lane's next action after its last one: pops the stack (leaving an instance
// when its marker comes up) until there is a node to visit or an instance to enter,
// but not past a marker or the end while leaves of the level are still pending.
template <bool ANY, bool SCENE, int W = 4>
__device__ __forceinline__ uint32_t nextState(const TraceParams& P, Stack& st, RayState& s, const Pending& q) {
    for (;;) {
        if (s.next != kNone) {
            if (SCENE && !s.inBlas && (s.next & kLeafBit)) return kStEnter;
            return q.n > pendingCap(W) - (uint32_t)W ? kStFlush : kStNode;
        }
        if (st.sp == 0) return q.n ? kStFlush : kStDone;
        if (SCENE && st.top() == kSentinel) {
            if (q.n) return kStFlush;
            st.pop();
            exactLevel(s.L, s.wo, s.wd);  // back to the top level
            s.lo = s.tmin;
            s.hi = (ANY || !s.found) ? s.tmax : s.best.t;
            s.nodes = P.target.nodes;
            s.fmt = P.target.fmt;
            s.inBlas = false;
            continue;
        }
        s.next = st.pop();
    }
}

// Persistent refill loop shared by the query kernels: each lane owns one work item
// (a ray). Every iteration the whole warp takes ONE kind of step, so that the node,
// leaf and instance-entry code paths do not run one after another in a warp:
//   LEAF  - lanes with pending leaves test them (when some lane must flush, or when at
//           least half the working lanes have leaves queued);
//   ENTER - lanes at a top-level leaf enter the instance (when at least a quarter of
//           the working lanes wait to, or no lane has a node to visit);
//   NODE  - lanes with a node to visit visit it, queueing the leaves they hit.
// Once the queue is exhausted and at most two lanes still work, each finishes its ray
// in a tight loop of single steps. (Speculative, leaf-deferring traversal after Aila
// and Laine, "Understanding the Efficiency of Ray Traversal on GPUs", HPG 2009.) When
// the warp's working lanes drop
// to P.refillBelow or fewer, idle lanes take fresh items from the global queue with one
// atomic per warp. Src supplies the items:
//   count()             number of items (may be read from device memory)
//   begin(i, P, st, s)  set up item i's ray in s; false if the item has no ray
//   finish(i, s)        consume item i's result s.best
// Any-hit queries (shadow and ambient-occlusion rays) take the per-ray form instead: with
// one copy of the leaf test per step it measured faster for them (terrain AO 0.758 ->
// 0.728 ms); closest hits keep the phased form (1M spheres 5.20 against 5.62 ms).
template <bool ANY, bool SCENE, bool COUNT, int FM = kFmMixed, class Src>
__device__ __forceinline__ void refillLoop(const TraceParams& P, Stack& st, Src& src) {
    if constexpr (ANY) {
        refillLoopPerRay<ANY, SCENE, COUNT, FM>(P, st, src);
        return;
    }
    constexpr int W = slotsOf(FM);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t ltMask = (1u << lane) - 1u;
    const unsigned long long total = src.count();
    RayState s;
    Visits v;
    Pending q{st.sh + st.shDepth * blockDim.x, 0};
    uint32_t item = kNone, state = kStDone;
    bool exhausted = false;
    for (;;) {
        uint32_t live = __ballot_sync(0xffffffffu, item != kNone);
        while (!exhausted && (uint32_t)__popc(live) <= P.refillBelow) {
            const uint32_t idle = ~live;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(P.counter, (unsigned long long)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base + __popc(idle) >= total) exhausted = true;
            if (item == kNone) {
                const unsigned long long mine = base + __popc(idle & ltMask);
                if (mine < total && src.begin((uint32_t)mine, P, st, s)) {
                    item = (uint32_t)mine;
                    if (COUNT) v = Visits{};
                    q.n = 0;
                    state = nextState<ANY, SCENE, W>(P, st, s, q);
                    if (state == kStDone) {  // nothing to traverse (an empty target)
                        src.finish(item, s);
                        if (COUNT) flushVisits(P.stats, v);
                        item = kNone;
                    }
                }
            }
            live = __ballot_sync(0xffffffffu, item != kNone);
        }
        if (live == 0) break;
        const bool on = item != kNone;
        const uint32_t b0 = __ballot_sync(0xffffffffu, on && (state & 1u));  // enter (working lanes)
        const uint32_t b1 = __ballot_sync(0xffffffffu, on && (state & 2u));  // flush
        const uint32_t queued = __ballot_sync(0xffffffffu, on && q.n > 0);
        const uint32_t flush = b1, enter = b0, node = live & ~(b0 | b1);
        const uint32_t working = (uint32_t)__popc(live);
        // the last rays of the warp (queue exhausted, at most two lanes working) run to
        // their end without votes, testing their leaves as soon as they are found
        const bool tail = exhausted && working <= 2u;
        uint32_t phase;
        if (flush || 2u * (uint32_t)__popc(queued) >= working)
            phase = kStFlush;
        else if (enter && (4u * (uint32_t)__popc(enter) >= working || !node))
            phase = kStEnter;
        else
            phase = kStNode;
        if (!on) continue;
        do {
        if (tail) phase = q.n ? kStFlush : state;
        bool acted = false;
        if (phase == kStFlush) {
            if (q.n) {
                acted = true;
                const uint32_t n = q.n;
                q.n = 0;
                for (uint32_t i = 0; i < n; ++i)
                    if (testLeaf<ANY, SCENE, COUNT>(P, s, q.at(i), &v) && ANY) break;
            }
        } else if (phase == kStEnter) {
            if (state == kStEnter) {
                acted = true;
                const uint32_t leaf = s.next & ~kLeafBit;
                s.next = kNone;
                enterInstance<ANY, COUNT>(P, st, s, reinterpret_cast<const InstanceRecord*>(P.target.leaves) + leaf,
                                          &v);
            }
        } else if (state == kStNode) {
            acted = true;
            visitNode<ANY, SCENE, COUNT, FM>(P, st, s, q, &v);
        }
        if (acted) state = (ANY && s.found) ? kStDone : nextState<ANY, SCENE, W>(P, st, s, q);
        } while (tail && state != kStDone);
        if (state == kStDone) {
            src.finish(item, s);
            if (COUNT) flushVisits(P.stats, v);
            item = kNone;
        }
    }
}

// Items = rays of a ray buffer; results = hit records.
template <bool SCENE>
struct RayBufferSource {
    uint32_t n;
    __device__ unsigned long long count() const { return n; }
    __device__ bool begin(uint32_t i, const TraceParams& P, Stack& st, RayState& s) const {
        const float4 a = P.rays[2 * (size_t)i], b = P.rays[2 * (size_t)i + 1];
        beginRay<SCENE>(P, st, s, f3(a), f3(b), a.w, b.w);
        return true;
    }
    const TraceParams* P;
    __device__ void finish(uint32_t i, const RayState& s) const { storeHit(P->hits, i, s.best); }
};

// Hit h of the ray (wo, wd, [tmin, tmax]): its t, u, v recomputed in double-float (kept when
// the FP64 test does not confirm the hit).
__device__ __forceinline__ void refineOne(const TraceParams& P, float3 wo, float3 wd, float tmin, float tmax, Hit& h) {
    if (h.prim == kInvalid) return;
    const bool scene = P.target.primType == kPrimScene;
    uint32_t primType, geomType;
    const void* leaves;
    const uint32_t* toLeaf;
    if (scene) {
        const InstanceRecord* R = P.sceneLeaves + P.scenePrimToLeaf[h.inst];
        primType = instPrimType(R->typeBits);
        geomType = instGeomType(R->typeBits);
        leaves = R->leaves;
        toLeaf = R->geometry->primToLeaf;
    } else {
        primType = P.target.primType;
        geomType = P.target.geomType;
        leaves = P.target.leaves;
        toLeaf = P.targetPrimToLeaf;
    }
    const float4* rec = nullptr;
    bool sphere = false;
    if (primType == GRT_PRIMITIVE_TRIANGLE_MESH) {
        rec = reinterpret_cast<const float4*>(leaves) + 3 * (size_t)toLeaf[h.prim];
    } else if (P.table && geomType < P.numGeomTypes) {
        const FuncEntry fe = P.table[(size_t)P.rayType * P.numGeomTypes + geomType];
        if (fe.func == GRT_INTERSECT_SPHERE) {
            rec = reinterpret_cast<const float4*>(fe.data) + h.prim;
            sphere = true;
        }
    }
    if (!rec) return;
    const float4* hi = nullptr;
    const float4* lo = nullptr;
    if (scene) {  // the instance's inverse frame: record rows plus their low parts
        const InstanceRecord* R = P.sceneLeaves + P.scenePrimToLeaf[h.inst];
        hi = R->inv;
        lo = P.fwd32 + kFrameRows * (size_t)h.inst + 3;
    }
    const float4 res = refineFF(hi, lo, wo, wd, rec, sphere, tmin, tmax);
    if (res.w != 0.f) h.t = res.x, h.u = res.y, h.v = res.z;
}

// The state of an all-hits walk of one ray on a per-thread stack of DEPTH entries: next()
// returns the ray's hits one at a time, in traversal order, each with t, u, v recomputed
// in double-float, then a record with prim == kInvalid. The stack points into the object, so
// an AllHitsWalk is used where it was begun and never copied.
template <int DEPTH, class U = NoUser>
struct AllHitsWalk {
    RayState s;
    uint32_t entries[DEPTH];
    Stack st;
    Hit buf[slotsOf(kFmMixed)];  // the hits of one visit
    int n, i;
    bool scene, finished;
    float3 o, d;
    float tmin, tmax;
    const U* user = nullptr;
    void* payload = nullptr;

    __device__ void begin(const TraceParams& P, float3 o_, float3 d_, float tmin_, float tmax_) {
        o = o_, d = d_, tmin = tmin_, tmax = tmax_;
        st = Stack{nullptr, entries, 0u, (uint32_t)DEPTH, 1u, 0u};
        scene = P.target.primType == kPrimScene;
        if (scene)
            beginRay<true>(P, st, s, o, d, tmin, tmax);
        else
            beginRay<false>(P, st, s, o, d, tmin, tmax);
        n = i = 0;
        finished = false;
        if (!scene && P.target.split) {  // each triangle sits in several leaves
            latchError(P.error, GRT_ERROR_INVALID_PARAMETER);
            finished = true;
        }
    }
    __device__ Hit next(const TraceParams& P) {
        while (i == n && !finished) {
            const int r = scene ? stepAll<true, U>(P, st, s, buf, user, payload)
                                : stepAll<false, U>(P, st, s, buf, user, payload);
            if (r < 0)
                finished = true;
            else
                n = r, i = 0;
        }
        if (i == n) return Hit{kInvalid, kInvalid, INFINITY, 0.f, 0.f};
        Hit h = buf[i++];
        refineOne(P, o, d, tmin, tmax, h);
        return h;
    }
    __device__ bool done() const { return finished && i == n; }
};

// Ray r's closest hit: t, u, v recomputed in double-float (the hit record is updated in place).
__device__ __forceinline__ void refineHit(const TraceParams& P, uint32_t r) {
    uint32_t* p = P.hits + 5 * (size_t)r;
    Hit h{p[0], p[1], __uint_as_float(p[2]), __uint_as_float(p[3]), __uint_as_float(p[4])};
    if (h.prim == kInvalid) return;
    const float4 a = P.rays[2 * (size_t)r], b = P.rays[2 * (size_t)r + 1];
    refineOne(P, f3(a), f3(b), a.w, b.w, h);
    p[2] = __float_as_uint(h.t);
    p[3] = __float_as_uint(h.u);
    p[4] = __float_as_uint(h.v);
}

}  // namespace grt
