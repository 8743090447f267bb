// Ray-query kernels (closest hit, any hit, fused ambient occlusion), ray generation
// (camera, ambient occlusion) and their host entry points. The traversal itself is in
// traverse.cuh.
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include <cmath>

#include "traverse.cuh"

namespace grt {

// FM: the node formats the walk may meet (traverse.cuh): kFmPlain (4-wide only),
// kFmQuant (4-wide or quantised, read per level) or kFmWide8 (8-wide on every level).
template <bool ANY, bool SCENE, bool COUNT, int FM = kFmPlain>
__global__ void traceKernel(TraceParams P) {
    extern __shared__ uint32_t sstack[];
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    Stack st{sstack + threadIdx.x, P.globalStack + gtid, P.sharedDepth, P.globalDepth, P.globalStride, 0};
    RayBufferSource<SCENE> src{P.count, &P};
    refillLoop<ANY, SCENE, COUNT, FM>(P, st, src);
}

// The closest hits' t, u, v recomputed in double-float, one thread per ray after traversal so
// that every lane of a warp takes part (FP64 is far slower than FP32 on this GPU).
// One thread per ray: the hit records are read with every load in flight at once, and
// the FP64 work of the hits (a few percent of the rays on a camera view) stays dense in
// the warps that have them.
static unsigned refineBlocks(uint32_t rays) { return std::max(1u, ceilDiv(rays, 256)); }

__global__ void __launch_bounds__(256) refineKernel(TraceParams P) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < P.count; r += gridDim.x * blockDim.x) refineHit(P, r);
}

// Every hit of each ray (Sec. 7.5): one thread per ray walks it on a local stack of
// kAllHitsDepth entries and stores its first maxHits hits (traversal order, refined in double-float)
// in hits[r * maxHits ...], the rest of the ray's slots as misses, and the number of
// hits found in counts[r].
constexpr int kAllHitsDepth = 96;

__global__ void __launch_bounds__(128) allHitsKernel(TraceParams P, uint32_t maxHits, uint32_t* counts) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.count) return;
    const float4 a = P.rays[2 * (size_t)r], b = P.rays[2 * (size_t)r + 1];
    AllHitsWalk<kAllHitsDepth> w;
    w.begin(P, f3(a), f3(b), a.w, b.w);
    uint32_t k = 0;
    uint32_t* out = P.hits + 5 * (size_t)r * maxHits;
    for (;;) {
        const Hit h = w.next(P);
        if (h.prim == kInvalid) break;
        if (k < maxHits) storeHit(out, k, h);
        ++k;
    }
    for (uint32_t j = k; j < maxHits; ++j) storeHit(out, j, Hit{kInvalid, kInvalid, INFINITY, 0.f, 0.f});
    counts[r] = k;
}

// ---------------------------------------------------------------- ambient occlusion (Sec. 4)
__global__ void aoRayKernel(const InstanceRecord* sceneLeaves, const uint32_t* scenePrimToLeaf, const float4* fwd32,
                            const float4* rays, const uint32_t* hits, uint32_t pixels, uint32_t spp,
                            unsigned long long seed, float length, float4* out) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pixels) return;
    AoFrame F;
    const bool ok = aoFrame(sceneLeaves, scenePrimToLeaf, fwd32, rays + 2 * (size_t)p, hits + 5 * (size_t)p, F);
    for (uint32_t s = 0; s < spp; ++s) {
        float4* o = out + 2 * ((size_t)p * spp + s);
        if (!ok) {
            o[0] = make_float4(0.f, 0.f, 0.f, 0.f);
            o[1] = make_float4(0.f, 0.f, 0.f, -1.f);
            continue;
        }
        const float3 dir = aoDirection(F, seed, p, s);
        o[0] = make_float4(F.org.x, F.org.y, F.org.z, 0.f);
        o[1] = make_float4(dir.x, dir.y, dir.z, length);
    }
}

// Fused ambient occlusion in three launches, with no ray buffer:
//  1. aoCompactKernel: pixels with a primary hit are appended to a list (one atomic
//     per warp) with their AO frames; every pixel's occlusion count starts at 0 (kept
//     in ao's words);
//  2. aoTraceKernel: the refill loop over the list's (pixel, sample) items; each
//     item's ray is generated in registers from the stored frame and traced as an
//     any-hit query, and an occluded sample adds 1 to its pixel's count;
//  3. aoFinishKernel: ao = count / samplesPerPixel for the listed pixels.
// Per listed hit pixel: its AO frame, computed once for all its samples, as 3 float4
// {org, valid}, {n, 0}, {tg, 0} (the bitangent n x tg is recomputed by the same
// operations, so the rays equal grtGenerateAORays's bit for bit).
__global__ void aoCompactKernel(TraceParams P, uint32_t pixels, uint32_t* __restrict__ list,
                                uint32_t* __restrict__ listCount, uint32_t* __restrict__ counts,
                                float4* __restrict__ frames) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool hit = p < pixels && P.primaryHits[5 * (size_t)p + 1] != kInvalid;
    if (p < pixels) counts[p] = 0u;
    const uint32_t mask = __ballot_sync(0xffffffffu, hit);
    const uint32_t lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0 && mask) base = atomicAdd(listCount, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!hit) return;
    const uint32_t slot = base + __popc(mask & ((1u << lane) - 1u));
    list[slot] = p;
    AoFrame F;
    const uint32_t* h = P.primaryHits + 5 * (size_t)p;
    const uint32_t valid =
        aoFrame(P.sceneLeaves, P.scenePrimToLeaf, P.fwd32, P.primaryRays + 2 * (size_t)p, h, F) ? 1u : kInvalid;
    frames[3 * (size_t)slot] = make_float4(F.org.x, F.org.y, F.org.z, __uint_as_float(valid));
    frames[3 * (size_t)slot + 1] = make_float4(F.n.x, F.n.y, F.n.z, 0.f);
    frames[3 * (size_t)slot + 2] = make_float4(F.tg.x, F.tg.y, F.tg.z, 0.f);
}

// Items = (listed pixel, sample); the ray comes from the pixel's stored frame.
struct AoSource {
    const TraceParams* P;
    const uint32_t* list;
    const uint32_t* listCount;
    uint32_t* counts;
    const float4* frames;
    __device__ unsigned long long count() const { return (unsigned long long)*listCount * P->spp; }
    __device__ bool begin(uint32_t i, const TraceParams& Pm, Stack& st, RayState& s) const {
        const uint32_t slot = i / Pm.spp, smp = i - slot * Pm.spp;
        const float4 a = frames[3 * (size_t)slot], b = frames[3 * (size_t)slot + 1], c = frames[3 * (size_t)slot + 2];
        if (__float_as_uint(a.w) == kInvalid) return false;  // not a triangle hit
        AoFrame F;
        F.org = f3(a), F.n = f3(b), F.tg = f3(c);
        F.bt = cross3(F.n, F.tg);
        beginRay<true>(Pm, st, s, F.org, aoDirection(F, Pm.seed, list[slot], smp), 0.0f, Pm.aoLength);
        return true;
    }
    __device__ void finish(uint32_t i, const RayState& s) const {
        if (s.best.prim != kInvalid) atomicAdd(&counts[list[i / P->spp]], 1u);
    }
};

// 96 registers: 5 blocks of 128 threads per SM instead of 4, 7% faster on the terrain
// AO workload despite a few spills (the closest-hit kernel is faster uncapped).
#ifndef GRT_AO_MAXNREG
#define GRT_AO_MAXNREG 96
#endif
template <bool COUNT, int FM = kFmPlain>
__global__ void __maxnreg__(GRT_AO_MAXNREG) aoTraceKernel(TraceParams P, const uint32_t* list, const uint32_t* listCount,
                                              uint32_t* counts, const float4* frames) {
    extern __shared__ uint32_t sstack[];
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    Stack st{sstack + threadIdx.x, P.globalStack + gtid, P.sharedDepth, P.globalDepth, P.globalStride, 0};
    AoSource src{&P, list, listCount, counts, frames};
    refillLoop<true, true, COUNT, FM>(P, st, src);
}

__global__ void aoFinishKernel(const uint32_t* __restrict__ list, const uint32_t* __restrict__ listCount,
                               uint32_t spp, float* ao) {
    const uint32_t n = *listCount;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t p = list[i];
        const uint32_t k = __float_as_uint(ao[p]);  // the occlusion count
        ao[p] = (float)k / (float)spp;
    }
}

// ---------------------------------------------------------------- Lambertian shading and its adjoint
// Per pixel with a primary hit on a triangle geometry: n_f = the face normal turned
// toward the viewer; s = max(0, n_f . l) with l used as given (the cosine law of Sec.
// 4.1; the Lambert BRDF c/pi of Sec. 5.2 with pi folded into the loss scale); V = 1
// unless the shadow ray from p + 1e-4 n_f along l (any hit, t in [0, inf)) is blocked;
// c(u,v) interpolates per-vertex colours; I = V s c(u,v), 0 for a miss.
//
// A scene is shaded the same way in world space: triangle (instance, prim) is triangle
// triOffset[instance] + prim of the object-space mesh (idx, pos, col), its vertices are
// mapped by the instance's forward frame (float32 rows), and the shadow ray is traced
// through the whole scene.
struct ShadeParams {
    const float4* rays;
    const uint32_t* hits;  // 5 words per pixel
    uint32_t n;
    const uint32_t* idx;   // 3 per triangle
    const float* pos;      // 3 per vertex
    const float* col;      // 3 per vertex
    const float* light;    // 3
    const uint32_t* triOffset;  // scenes: first triangle of each instance ID's mesh
    const float4* frames;       // scenes: kFrameRows float4 per instance ID (forward frame rows 0-2)
    const InstanceRecord* sceneLeaves;  // scenes: instance records (to skip custom-primitive instances)
    const uint32_t* scenePrimToLeaf;
    float* image;          // 3 per pixel, or null (visibility only)
    uint8_t* vis;          // per pixel, or null
    const float* gimg;     // adjoint: dL/dI, 3 per pixel
    float* gcol;
    float* glight;
    float* gpos;
};

struct ShadeHit {
    float3 v0, v1, v2, o, d, nf;  // vertices in world space
    float nl, u, v, t;
    uint32_t i0, i1, i2;
    float4 m0, m1, m2;  // scenes: the instance's forward frame rows
};

__device__ __forceinline__ float3 ld3(const float* p, uint32_t k) { return make_float3(p[3 * k], p[3 * k + 1], p[3 * k + 2]); }

// Frame row applied to an object-space point: m.xyz . a + m.w.
__device__ __forceinline__ float frameRow(float4 m, float3 a) { return fmaf(m.x, a.x, fmaf(m.y, a.y, fmaf(m.z, a.z, m.w))); }

// Whether the hit record h names a shaded triangle: a hit at all, and in a scene one on
// a triangle-mesh instance (hits on custom primitives are occluders only, image 0).
template <bool SCENE>
__device__ __forceinline__ bool shadedHit(const ShadeParams& S, const uint32_t* h) {
    if (h[1] == kInvalid) return false;
    if (!SCENE) return true;
    return instPrimType(S.sceneLeaves[S.scenePrimToLeaf[h[0]]].typeBits) == GRT_PRIMITIVE_TRIANGLE_MESH;
}

template <bool SCENE>
__device__ __forceinline__ ShadeHit shadeSetup(const ShadeParams& S, float4 ra, float4 rb, uint32_t inst, uint32_t prim,
                                               float t, float u, float v, float3 l) {
    ShadeHit H;
    const size_t tri = SCENE ? (size_t)S.triOffset[inst] + prim : (size_t)prim;
    H.i0 = S.idx[3 * tri], H.i1 = S.idx[3 * tri + 1], H.i2 = S.idx[3 * tri + 2];
    H.v0 = ld3(S.pos, H.i0), H.v1 = ld3(S.pos, H.i1), H.v2 = ld3(S.pos, H.i2);
    if (SCENE) {
        const float4* F = S.frames + kFrameRows * (size_t)inst;
        H.m0 = F[0], H.m1 = F[1], H.m2 = F[2];
        H.v0 = make_float3(frameRow(H.m0, H.v0), frameRow(H.m1, H.v0), frameRow(H.m2, H.v0));
        H.v1 = make_float3(frameRow(H.m0, H.v1), frameRow(H.m1, H.v1), frameRow(H.m2, H.v1));
        H.v2 = make_float3(frameRow(H.m0, H.v2), frameRow(H.m1, H.v2), frameRow(H.m2, H.v2));
    }
    H.o = f3(ra), H.d = f3(rb);
    float3 n = normalize3(cross3(H.v1 - H.v0, H.v2 - H.v0));
    if (dot3(n, H.d) > 0.0f) n = n * -1.0f;
    H.nf = n;
    H.nl = dot3(n, l);
    H.t = t, H.u = u, H.v = v;
    return H;
}

__device__ __forceinline__ float3 shadeColour(const ShadeParams& S, const ShadeHit& H) {
    const float w0 = 1.0f - H.u - H.v;
    const float3 c0 = ld3(S.col, H.i0), c1 = ld3(S.col, H.i1), c2 = ld3(S.col, H.i2);
    return make_float3(w0 * c0.x + H.u * c1.x + H.v * c2.x, w0 * c0.y + H.u * c1.y + H.v * c2.y,
                       w0 * c0.z + H.u * c1.z + H.v * c2.z);
}

// Items = pixels; a lit hit pixel traces its shadow ray, everything else is written at once.
template <bool SCENE>
struct ShadowSource {
    const ShadeParams* S;
    __device__ unsigned long long count() const { return S->n; }
    __device__ ShadeHit setup(uint32_t i) const {
        const uint32_t* h = S->hits + 5 * (size_t)i;
        const float3 l = make_float3(S->light[0], S->light[1], S->light[2]);
        return shadeSetup<SCENE>(*S, S->rays[2 * (size_t)i], S->rays[2 * (size_t)i + 1], h[0], h[1],
                                 __uint_as_float(h[2]), __uint_as_float(h[3]), __uint_as_float(h[4]), l);
    }
    __device__ bool begin(uint32_t i, const TraceParams& P, Stack& st, RayState& s) const {
        if (shadedHit<SCENE>(*S, S->hits + 5 * (size_t)i)) {
            const ShadeHit H = setup(i);
            if (H.nl > 0.0f) {
                const float3 l = make_float3(S->light[0], S->light[1], S->light[2]);
                beginRay<SCENE>(P, st, s, (H.o + H.d * H.t) + H.nf * 1e-4f, l, 0.0f, INFINITY);
                return true;
            }
        }
        if (S->image) S->image[3 * (size_t)i] = 0.f, S->image[3 * (size_t)i + 1] = 0.f, S->image[3 * (size_t)i + 2] = 0.f;
        if (S->vis) S->vis[i] = 1;
        return false;
    }
    __device__ void finish(uint32_t i, const RayState& s) const {
        const float V = s.best.prim == kInvalid ? 1.0f : 0.0f;
        if (S->image) {
            const ShadeHit H = setup(i);
            const float3 c = shadeColour(*S, H);
            const float k = V * H.nl;
            S->image[3 * (size_t)i] = k * c.x, S->image[3 * (size_t)i + 1] = k * c.y, S->image[3 * (size_t)i + 2] = k * c.z;
        }
        if (S->vis) S->vis[i] = (uint8_t)V;
    }
};

template <bool SCENE, int FM = kFmPlain>
__global__ void shadeForwardKernel(TraceParams P, ShadeParams S) {
    extern __shared__ uint32_t sstack[];
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    Stack st{sstack + threadIdx.x, P.globalStack + gtid, P.sharedDepth, P.globalDepth, P.globalStride, 0};
    ShadowSource<SCENE> src{&S};
    refillLoop<true, SCENE, false, FM>(P, st, src);
}

// One pixel's share of the adjoint: dL/dc_k and dL/dv_k for the hit triangle's three
// vertices, and its term of dL/dl. live = false for a miss, an unlit or a shadowed pixel.
struct PixelAdjoint {
    bool live;
    uint32_t prim;
    uint32_t vk[3];
    float3 dc[3], dv[3];
    float3 dl;
};

template <bool SCENE>
__device__ __forceinline__ PixelAdjoint pixelAdjoint(const ShadeParams& S, uint32_t i, float3 l) {
    PixelAdjoint A;
    A.live = false;
    const uint32_t* h = S.hits + 5 * (size_t)i;
    if (!shadedHit<SCENE>(S, h)) return A;  // a miss reads nothing else
    const uint32_t prim = h[1];
    const float t = __uint_as_float(h[2]), u = __uint_as_float(h[3]), v = __uint_as_float(h[4]);
    const float4 ra = S.rays[2 * (size_t)i], rb = S.rays[2 * (size_t)i + 1];
    const ShadeHit H = shadeSetup<SCENE>(S, ra, rb, h[0], prim, t, u, v, l);
    if (!(H.nl > 0.0f)) return A;  // unlit: I = 0 and no gradient
    const float V = S.vis ? (float)S.vis[i] : 1.0f;
    if (V == 0.0f) return A;
    const float3 g = make_float3(S.gimg[3 * (size_t)i], S.gimg[3 * (size_t)i + 1], S.gimg[3 * (size_t)i + 2]);
    const float w[3] = {1.0f - u - v, u, v};
    const float s = H.nl;
    A.live = true;
    A.prim = prim;
    A.vk[0] = H.i0, A.vk[1] = H.i1, A.vk[2] = H.i2;
    // colours: dI/dc_k = s w_k per channel
#pragma unroll
    for (int k = 0; k < 3; ++k) A.dc[k] = g * (s * w[k]);
    const float3 c0 = ld3(S.col, H.i0), c1 = ld3(S.col, H.i1), c2 = ld3(S.col, H.i2);
    const float3 c = make_float3(w[0] * c0.x + u * c1.x + v * c2.x, w[0] * c0.y + u * c1.y + v * c2.y,
                                 w[0] * c0.z + u * c1.z + v * c2.z);
    const float gs = dot3(g, c);
    A.dl = H.nf * gs;  // light, where lit
    // positions through the face normal: m = e1 x e2, n = m / |m|, n_f = sigma n
    const float3 e1 = H.v1 - H.v0, e2 = H.v2 - H.v0;
    const float3 m = cross3(e1, e2);
    const float ml = sqrtf(dot3(m, m));
    const float3 n = m * (1.0f / ml);
    const float sigma = dot3(H.nf, n) > 0.f ? 1.f : -1.f;
    const float3 gm = (l - n * dot3(n, l)) * (gs * sigma / ml);
    A.dv[0] = cross3(e1 - e2, gm), A.dv[1] = cross3(e2, gm), A.dv[2] = cross3(gm, e1);
    // positions through the barycentrics on the fixed ray: d(t,u,v)/dv_k = -w_k A^-1, A = [-d | e1 | e2]
    const float gu = s * dot3(g, c1 - c0), gv = s * dot3(g, c2 - c0);
    const float3 nd = H.d * -1.0f;
    const float det = dot3(nd, m);
    if (det != 0.0f) {
        const float3 y = (cross3(e2, nd) * gu + cross3(nd, e1) * gv) * (1.0f / det);
#pragma unroll
        for (int k = 0; k < 3; ++k) A.dv[k] = A.dv[k] - y * w[k];
    }
    if (SCENE) {  // world vertex = M a + T: dL/da = M^T dL/dv
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float3 g = A.dv[k];
            A.dv[k] = make_float3(H.m0.x * g.x + H.m1.x * g.y + H.m2.x * g.z, H.m0.y * g.x + H.m1.y * g.y + H.m2.y * g.z,
                                  H.m0.z * g.x + H.m1.z * g.y + H.m2.z * g.z);
        }
    }
    return A;
}

// Sum of x over lanes [lane, end] of a run of consecutive lanes (end = the run's last lane).
__device__ __forceinline__ float runSum(float x, uint32_t lane, uint32_t end) {
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const float y = __shfl_down_sync(0xffffffffu, x, o);
        if (lane + o <= end) x += y;
    }
    return x;
}

__device__ __forceinline__ float3 runSum3(float3 x, uint32_t lane, uint32_t end) {
    return make_float3(runSum(x.x, lane, end), runSum(x.y, lane, end), runSum(x.z, lane, end));
}

// Adds one vertex's 3-vector into a block-private shared copy when there is one and the
// vertex is inside it, else into the output in global memory.
template <bool PRIV>
__device__ __forceinline__ void addVertex3(float* priv, float* out, uint32_t nv, uint32_t k, float3 g) {
    if (PRIV && k < nv) {
        atomicAdd(priv + 3 * k, g.x), atomicAdd(priv + 3 * k + 1, g.y), atomicAdd(priv + 3 * k + 2, g.z);
    } else {
        atomicAdd(out + 3 * (size_t)k, g.x), atomicAdd(out + 3 * (size_t)k + 1, g.y),
            atomicAdd(out + 3 * (size_t)k + 2, g.z);
    }
}

// Warp-wide scatter of the vertex gradients (all 32 lanes call it). Neighbouring pixels
// mostly hit the same triangle: each run of consecutive lanes with the same triangle is
// summed by shuffles and its first lane adds the sums (18 atomics per run, not per pixel).
template <bool PRIV>
__device__ __forceinline__ void scatterAdjoint(const PixelAdjoint& A, float* priv, const ShadeParams& S, uint32_t nv) {
    const unsigned full = 0xffffffffu;
    if (!__any_sync(full, A.live)) return;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t key = A.live ? A.prim : kInvalid;
    const uint32_t next = __shfl_down_sync(full, key, 1), prev = __shfl_up_sync(full, key, 1);
    const unsigned ends = __ballot_sync(full, lane == 31u || next != key);
    const uint32_t end = (uint32_t)__ffs(ends & (full << lane)) - 1u;
    const bool head = lane == 0u || prev != key;
    float3 dc[3], dv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dc[k] = runSum3(A.live ? A.dc[k] : make_float3(0.f, 0.f, 0.f), lane, end);
        dv[k] = runSum3(A.live ? A.dv[k] : make_float3(0.f, 0.f, 0.f), lane, end);
    }
    if (head && A.live) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            addVertex3<PRIV>(priv, S.gcol, nv, A.vk[k], dc[k]);
            addVertex3<PRIV>(priv + 3 * nv, S.gpos, nv, A.vk[k], dv[k]);
        }
    }
}

// Adjoint: blocks take tiles of consecutive pixels (image rows) from a work counter;
// one thread per pixel, reading the stored hit records and visibility. With PRIV the
// colour and position gradients of every vertex (6 floats each) are summed in shared
// memory and each block adds its nonzero entries to the output once at the end: a small
// mesh's gradients sit in a few hundred cache lines, and per-pixel global atomics on
// them queue in a few L2 slices.
template <bool SCENE, bool PRIV>
__global__ void shadeBackwardKernel(TraceParams P, ShadeParams S, uint32_t nv) {
    extern __shared__ uint32_t sstack[];
    __shared__ unsigned long long tile;
    float* priv = reinterpret_cast<float*>(sstack);
    if (PRIV)
        for (uint32_t j = threadIdx.x; j < 6 * nv; j += blockDim.x) priv[j] = 0.0f;
    const float3 l = make_float3(S.light[0], S.light[1], S.light[2]);
    float3 gl = make_float3(0.f, 0.f, 0.f);
    const uint32_t perTile = blockDim.x * 8u;
    for (;;) {
        if (threadIdx.x == 0) tile = atomicAdd(P.counter, 1ull);
        __syncthreads();  // also orders the zeroing of priv before the first adds
        const unsigned long long first = tile * perTile;
        __syncthreads();  // every thread has read tile before thread 0 takes the next one
        if (first >= S.n) break;
        for (uint32_t k = threadIdx.x; k < perTile; k += blockDim.x) {  // same trip count in every lane
            PixelAdjoint A;
            A.live = false;
            if (first + k < S.n) A = pixelAdjoint<SCENE>(S, (uint32_t)(first + k), l);
            if (A.live) gl = gl + A.dl;
            scatterAdjoint<PRIV>(A, priv, S, nv);
        }
    }
    // light gradient: warp sum, one atomic per warp and axis
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gl.x += __shfl_xor_sync(0xffffffffu, gl.x, o);
        gl.y += __shfl_xor_sync(0xffffffffu, gl.y, o);
        gl.z += __shfl_xor_sync(0xffffffffu, gl.z, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&S.glight[0], gl.x);
        atomicAdd(&S.glight[1], gl.y);
        atomicAdd(&S.glight[2], gl.z);
    }
    if (PRIV) {
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < 3 * nv; j += blockDim.x) {
            const float a = priv[j], b = priv[3 * nv + j];
            if (a != 0.0f) atomicAdd(&S.gcol[j], a);
            if (b != 0.0f) atomicAdd(&S.gpos[j], b);
        }
    }
}

// ---------------------------------------------------------------- camera rays (Sec. 3.2)
__global__ void cameraRayKernel(grtCamera cam, uint32_t W, uint32_t H, float4* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    const uint32_t x = i % W, y = i / W;
    const float3 o = make_float3(cam.origin[0], cam.origin[1], cam.origin[2]);
    const float3 right = make_float3(cam.right[0], cam.right[1], cam.right[2]);
    const float3 up = make_float3(cam.up[0], cam.up[1], cam.up[2]);
    const float3 fwd = normalize3(cross3(up, right));
    const float u = ((float)x + 0.5f) / (float)W, v = ((float)y + 0.5f) / (float)H;
    // lerp(-right, right, u) + lerp(up, -up, v)
    const float3 to = o + fwd + right * (2.0f * u - 1.0f) + up * (1.0f - 2.0f * v);
    const float3 d = normalize3(to - o);
    out[2 * (size_t)i] = make_float4(o.x, o.y, o.z, 0.0f);
    out[2 * (size_t)i + 1] = make_float4(d.x, d.y, d.z, INFINITY);
}

// Uniform random rays: origin uniform in the box [lo, hi], direction uniform on the unit
// sphere (Archimedes: z uniform in [-1, 1], azimuth uniform), from the splitmix64
// numbers of stream `seed` at ray i's counters (samples 0..2, dims 0..1). The radius
// sqrt(1 - z^2) is evaluated as 2 sqrt(xi (1 - xi)), the same real number: 1 - xi is
// exact for a multiple of 2^-24, where 1 - z*z cancels near the poles.
__global__ void uniformRayKernel(float3 lo, float3 ext, uint64_t seed, uint32_t n, float tmin, float tmax,
                                 float4* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ox = sampleXi(seed, i, 0, 0), oy = sampleXi(seed, i, 0, 1), oz = sampleXi(seed, i, 1, 0);
    const float xz = sampleXi(seed, i, 1, 1), xp = sampleXi(seed, i, 2, 0);
    const float z = 1.0f - 2.0f * xz;
    const float r = 2.0f * sqrtf(xz * (1.0f - xz));
    float sn, cs;
    sincospif(2.0f * xp, &sn, &cs);
    out[2 * (size_t)i] = make_float4(fmaf(ext.x, ox, lo.x), fmaf(ext.y, oy, lo.y), fmaf(ext.z, oz, lo.z), tmin);
    out[2 * (size_t)i + 1] = make_float4(r * cs, r * sn, z, tmax);
}

// ---------------------------------------------------------------- host side
struct LaunchShape {
    int blockSize;
    int blocks;
};

template <class K>
static LaunchShape persistentShape(Context* c, K kernel, int blockSize, size_t smem) {
    static std::mutex m;
    static std::unordered_map<size_t, int> cache;
    const size_t key = ((size_t)(void*)kernel) ^ ((size_t)blockSize << 48) ^ (smem << 20);
    int perSm = 0;
    {
        std::lock_guard<std::mutex> g(m);
        auto it = cache.find(key);
        if (it != cache.end()) perSm = it->second;
    }
    if (perSm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSm, kernel, blockSize, smem) != cudaSuccess || perSm < 1)
            perSm = 1;
        std::lock_guard<std::mutex> g(m);
        cache[key] = perSm;
    }
    return LaunchShape{blockSize, perSm * smCount(c)};
}

static grtError resolveOptions(const grtTraceOptions* opt, int* blockSize, uint32_t* sh, uint32_t* gl) {
    *blockSize = (opt && opt->blockSize) ? (int)opt->blockSize : 128;
    *sh = (opt && opt->sharedStackDepth) ? opt->sharedStackDepth : 16u;
    *gl = (opt && opt->globalStackDepth) ? opt->globalStackDepth : 64u;
    if (*blockSize != 64 && *blockSize != 128 && *blockSize != 256) return GRT_ERROR_INVALID_PARAMETER;
    if (*sh < 1 || *sh > 32 || *gl > 4096) return GRT_ERROR_INVALID_PARAMETER;
    if (opt && (opt->flags & ~GRT_TRACE_FLAG_COUNT)) return GRT_ERROR_INVALID_PARAMETER;
    return GRT_SUCCESS;
}

// Everything a launch needs except the kernel-specific fields.
// defaultCompact: the refill threshold when the options leave it 0 (measured best per
// query kind: 0.5 for closest / any hit and shading, 0.6 for fused ambient occlusion).
static grtError prepareTrace(Context* c, grtScene scene, grtGeometry geom, grtFuncTable table,
                             const grtTraceOptions* opt, TraceParams& P, bool* isScene, int* blockSize,
                             float defaultCompact = 0.5f) {
    if ((scene != nullptr) == (geom != nullptr)) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = findBvh(scene ? (const void*)scene : (const void*)geom);
    if (!o) return GRT_ERROR_INVALID_PARAMETER;
    if (scene && o->primType != kPrimScene) return GRT_ERROR_INVALID_PARAMETER;
    if (geom && o->primType == kPrimScene) return GRT_ERROR_INVALID_PARAMETER;
    if (!o->built) return GRT_ERROR_NOT_BUILT;
    *isScene = scene != nullptr;
    P.target.nodes = (const float4*)(o->qnodes ? o->qnodes : o->w8nodes ? o->w8nodes : o->wide);
    P.target.fmt = o->qnodes ? 1u : o->w8nodes ? 2u : 0u;
    P.target.split = o->split ? 1u : 0u;
    P.target.leaves = o->leaves;
    P.target.primType = o->primType;
    P.target.geomType = o->geomType;
    P.target.empty = o->primCount == 0;
    P.maxSteps = 1u << 26;  // far above any legitimate walk; stops a corrupted (cyclic) hierarchy
    P.rayMask = (opt && opt->rayMask) ? opt->rayMask : 0xFFFFFFFFu;
    const float compact = (opt && opt->compactThreshold > 0.f) ? fminf(opt->compactThreshold, 1.f) : defaultCompact;
    P.refillBelow = (uint32_t)(compact * 32.f);
    P.inv64 = o->inv64;
    P.fwd32 = (const float4*)o->fwd32;
    if (scene) {
        P.sceneLeaves = (const InstanceRecord*)o->leaves;
        P.scenePrimToLeaf = o->primToLeaf;
    } else {
        P.targetPrimToLeaf = o->primToLeaf;
    }
    if (table) {
        FuncTableObject* t = findFuncTable(table);
        if (!t) return GRT_ERROR_INVALID_PARAMETER;
        if (t->userEntries) {  // user code runs only in kernels that trace through grt_device.cuh
            logf(GRT_LOG_ERROR, "the function table names user functions; trace through grt_device.cuh");
            return GRT_ERROR_INVALID_PARAMETER;
        }
        P.table = t->dEntries;
        P.numGeomTypes = t->numGeomTypes;
        P.rayType = opt ? opt->rayType : 0u;
        if (P.rayType >= t->numRayTypes) return GRT_ERROR_INVALID_PARAMETER;
    }
    uint32_t sh, gl;
    grtError e = resolveOptions(opt, blockSize, &sh, &gl);
    if (e != GRT_SUCCESS) return e;
    P.sharedDepth = sh;
    P.globalDepth = gl;
    P.error = &workspace(c)->error;
    P.stats = workspace(c)->stats;
    return GRT_SUCCESS;
}

// Global stack for `threads` threads (the caller's buffer or the context's scratch),
// plus optionally `extraBytes` more of context scratch returned in *extra.
static grtError bindGlobalStack(Context* c, const grtTraceOptions* opt, int threads, TraceParams& P,
                                size_t extraBytes = 0, void** extra = nullptr) {
    const size_t need = alignUp((size_t)threads * P.globalDepth * sizeof(uint32_t), 256);
    P.globalStride = (uint32_t)threads;
    void* p = nullptr;
    if (opt && opt->globalStack) {
        if (opt->globalStackBytes < need) return GRT_ERROR_INVALID_PARAMETER;
        P.globalStack = (uint32_t*)opt->globalStack;
        if (!extraBytes) return GRT_SUCCESS;
        grtError e = contextScratch(c, extraBytes, &p);
        *extra = p;
        return e;
    }
    grtError e = contextScratch(c, std::max<size_t>(need + extraBytes, 256), &p);
    P.globalStack = (uint32_t*)p;
    if (extraBytes) *extra = static_cast<char*>(p) + need;
    return e;
}

// The node formats a walk over P's target can meet (the kernel variant to launch): a
// geometry's own format; an 8-wide scene walks 8-wide levels only (its instances must be
// 8-wide); a 4-wide scene walks the 4-wide or quantised nodes of its instances, and can
// meet quantised ones only while such a geometry exists (a scene instances live
// geometries only).
static int walkFormats(const TraceParams& P, bool scene) {
    if (P.target.fmt == 2) return kFmWide8;
    if (P.target.fmt == 1 || (scene && anyQuantGeometry())) return kFmQuant;
    return kFmPlain;
}

template <bool ANY, bool COUNT>
static void traceKernelFor(bool scene, int fm, void (**k)(TraceParams)) {
    if (fm == kFmWide8)
        *k = scene ? traceKernel<ANY, true, COUNT, kFmWide8> : traceKernel<ANY, false, COUNT, kFmWide8>;
    else if (fm == kFmQuant)
        *k = scene ? traceKernel<ANY, true, COUNT, kFmQuant> : traceKernel<ANY, false, COUNT, kFmQuant>;
    else
        *k = scene ? traceKernel<ANY, true, COUNT> : traceKernel<ANY, false, COUNT>;
}

template <bool ANY>
static grtError launchTrace(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, uint32_t n,
                            grtHit* hits, grtFuncTable table, const grtTraceOptions* opt, void* stream) {
    if (!ctx) return GRT_ERROR_INVALID_PARAMETER;
    if (n && (!rays || !hits || ((uintptr_t)rays & 15))) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    TraceParams P{};
    bool isScene = false;
    int bs = 128;
    grtError e = prepareTrace(c, scene, geom, table, opt, P, &isScene, &bs);
    if (e != GRT_SUCCESS || n == 0) return e;
    const bool count = opt && (opt->flags & GRT_TRACE_FLAG_COUNT);
    P.rays = (const float4*)rays;
    P.hits = (uint32_t*)hits;
    P.count = n;
    void (*kernel)(TraceParams) = nullptr;
    if (count)
        traceKernelFor<ANY, true>(isScene, walkFormats(P, isScene), &kernel);
    else
        traceKernelFor<ANY, false>(isScene, walkFormats(P, isScene), &kernel);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = (size_t)bs * traceSmemWords(P.sharedDepth, slotsOf(walkFormats(P, isScene))) * sizeof(uint32_t);
    LaunchShape L = persistentShape(c, kernel, bs, smem);
    L.blocks = std::min<int>(L.blocks, (int)ceilDiv(n, bs));
    e = bindGlobalStack(c, opt, L.blocks * bs, P);
    if (e != GRT_SUCCESS) return e;
    P.counter = nextCounter(c);
    GRT_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));
    kernel<<<L.blocks, bs, smem, s>>>(P);
    if (!ANY) refineKernel<<<refineBlocks(n), 256, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    noteLaunches(ANY ? 1 : 2);
    return GRT_SUCCESS;
}

// ---------------------------------------------------------------- allocation-free closest hit
// Scratch of grtTraceClosestNoAlloc, resident on every device that loads the library:
// bytes [0, 256) hold the work counter, the rest the traversal's global stack.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr size_t kNoAllocStackOffset = 256;
static __device__ __align__(256) unsigned char g_noAllocScratch[kNoAllocScratchBytes];

static std::mutex g_noAllocMutex;
static std::unordered_map<int, void*> g_noAllocAddress;  // device ordinal -> device address of the array

// Device address of the scratch array on the current device. Host code cannot use the
// array's name as an address (it names a host-side stand-in), so the address is
// looked up once per device with that device current and cached.
static grtError noAllocScratchAddress(int device, void** out) {
    std::lock_guard<std::mutex> g(g_noAllocMutex);
    auto it = g_noAllocAddress.find(device);
    if (it != g_noAllocAddress.end()) {
        *out = it->second;
        return GRT_SUCCESS;
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noAllocScratch);
    if (e != cudaSuccess || p == nullptr) {
        logf(GRT_LOG_ERROR, "grtTraceClosestNoAlloc: scratch address lookup failed: %s", cudaGetErrorString(e));
        return GRT_ERROR_CUDA;
    }
    g_noAllocAddress[device] = p;
    *out = p;
    return GRT_SUCCESS;
}

}  // namespace grt

using namespace grt;

extern "C" {

grtError grtTraceClosestNoAlloc(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays,
                                uint32_t rayCount, grtHit* hits, grtFuncTable table, const grtTraceOptions* options,
                                void* stream) {
    if (!ctx) return GRT_ERROR_INVALID_PARAMETER;
    if (rayCount && (!rays || !hits || ((uintptr_t)rays & 15))) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    int device = -1;
    GRT_CUDA(cudaGetDevice(&device));
    if (device != deviceOf(c)) return GRT_ERROR_INVALID_PARAMETER;
    TraceParams P{};
    bool isScene = false;
    int bs = 128;
    grtError e = prepareTrace(c, scene, geom, table, options, P, &isScene, &bs);
    if (e != GRT_SUCCESS || rayCount == 0) return e;
    // the grid keeps at least one block per SM (fewer only when there are fewer rays)
    const size_t capacity = kNoAllocScratchBytes - kNoAllocStackOffset;
    const size_t perBlock = (size_t)bs * P.globalDepth * sizeof(uint32_t);
    const size_t minBlocks = std::min<size_t>((size_t)smCount(c), ceilDiv(rayCount, bs));
    if (perBlock * minBlocks > capacity) {
        logf(GRT_LOG_ERROR,
             "grtTraceClosestNoAlloc: %zu blocks of %d threads with globalStackDepth %u need %zu bytes of global "
             "stack, more than the %zu-byte static scratch",
             minBlocks, bs, P.globalDepth, perBlock * minBlocks, capacity);
        return GRT_ERROR_INVALID_PARAMETER;
    }
    void* base = nullptr;
    e = noAllocScratchAddress(device, &base);
    if (e != GRT_SUCCESS) return e;
    const bool count = options && (options->flags & GRT_TRACE_FLAG_COUNT);
    P.rays = (const float4*)rays;
    P.hits = (uint32_t*)hits;
    P.count = rayCount;
    void (*kernel)(TraceParams) = nullptr;
    if (count)
        traceKernelFor<false, true>(isScene, walkFormats(P, isScene), &kernel);
    else
        traceKernelFor<false, false>(isScene, walkFormats(P, isScene), &kernel);
    const size_t smem = (size_t)bs * traceSmemWords(P.sharedDepth, slotsOf(walkFormats(P, isScene))) * sizeof(uint32_t);
    LaunchShape L = persistentShape(c, kernel, bs, smem);
    L.blocks = std::min<int>(L.blocks, (int)ceilDiv(rayCount, bs));
    L.blocks = std::max(1, std::min<int>(L.blocks, (int)(capacity / perBlock)));  // the grid shrinks to fit
    P.counter = reinterpret_cast<unsigned long long*>(base);
    P.globalStack = reinterpret_cast<uint32_t*>(static_cast<char*>(base) + kNoAllocStackOffset);
    P.globalStride = (uint32_t)(L.blocks * bs);
    cudaStream_t s = (cudaStream_t)stream;
    GRT_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));  // the work counter starts at zero
    kernel<<<L.blocks, bs, smem, s>>>(P);
    refineKernel<<<refineBlocks(rayCount), 256, 0, s>>>(P);
    GRT_LAUNCH_CHECK();
    noteLaunches(2);
    return GRT_SUCCESS;
}

grtError grtGetTraceGlobalStackSize(grtContext ctx, const grtTraceOptions* options, size_t* sizeBytes) {
    if (!ctx || !sizeBytes) return GRT_ERROR_INVALID_PARAMETER;
    int bs;
    uint32_t sh, gl;
    grtError e = resolveOptions(options, &bs, &sh, &gl);
    if (e != GRT_SUCCESS) return e;
    Context* c = asContext(ctx);
    int threads = 0;
    // every variant a launch may choose, each with its own shared memory
    auto most = [&](auto k, int w) {
        const size_t sm = (size_t)bs * traceSmemWords(sh, w) * sizeof(uint32_t);
        threads = std::max(threads, persistentShape(c, k, bs, sm).blocks * bs);
    };
    most(traceKernel<false, false, false>, 4), most(traceKernel<false, true, false>, 4);
    most(traceKernel<true, false, false>, 4), most(traceKernel<true, true, false>, 4);
    most(traceKernel<false, false, true>, 4), most(traceKernel<false, true, true>, 4);
    most(traceKernel<true, false, true>, 4), most(traceKernel<true, true, true>, 4);
    most(traceKernel<false, false, false, kFmWide8>, 8), most(traceKernel<false, true, false, kFmWide8>, 8);
    most(traceKernel<true, false, false, kFmWide8>, 8), most(traceKernel<true, true, false, kFmWide8>, 8);
    most(traceKernel<false, false, true, kFmWide8>, 8), most(traceKernel<false, true, true, kFmWide8>, 8);
    most(traceKernel<true, false, true, kFmWide8>, 8), most(traceKernel<true, true, true, kFmWide8>, 8);
    most(traceKernel<false, false, false, kFmQuant>, 4), most(traceKernel<false, true, false, kFmQuant>, 4);
    most(traceKernel<true, false, false, kFmQuant>, 4), most(traceKernel<true, true, false, kFmQuant>, 4);
    most(traceKernel<false, false, true, kFmQuant>, 4), most(traceKernel<false, true, true, kFmQuant>, 4);
    most(traceKernel<true, false, true, kFmQuant>, 4), most(traceKernel<true, true, true, kFmQuant>, 4);
    most(aoTraceKernel<false>, 4), most(aoTraceKernel<true>, 4);
    most(aoTraceKernel<false, kFmWide8>, 8), most(aoTraceKernel<true, kFmWide8>, 8);
    most(aoTraceKernel<false, kFmQuant>, 4), most(aoTraceKernel<true, kFmQuant>, 4);
    *sizeBytes = (size_t)threads * gl * sizeof(uint32_t);
    return GRT_SUCCESS;
}

grtError grtGetDeviceTarget(grtContext ctx, grtScene scene, grtGeometry geom, grtFuncTable table, uint32_t rayType,
                            grtDeviceTarget* out) {
    if (!ctx || !out || (scene != nullptr) == (geom != nullptr)) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = findBvh(scene ? (const void*)scene : (const void*)geom);
    if (!o || (scene != nullptr) != (o->primType == kPrimScene)) return GRT_ERROR_INVALID_PARAMETER;
    if (!o->built) return GRT_ERROR_NOT_BUILT;
    grtDeviceTarget t{};
    t.nodes = o->qnodes ? o->qnodes : o->w8nodes ? o->w8nodes : o->wide;
    t.nodeFormat = (o->qnodes ? 1u : o->w8nodes ? 2u : 0u) | (o->split ? 0x100u : 0u);
    t.leaves = o->leaves;
    t.primToLeaf = o->primToLeaf;
    t.frames64 = o->inv64;
    t.frames32 = o->fwd32;
    t.deviceError = &workspace(asContext(ctx))->error;
    t.primType = o->primType;
    t.geomType = o->geomType;
    t.primCount = o->primCount;
    t.rayType = rayType;
    if (table) {
        FuncTableObject* f = findFuncTable(table);
        if (!f || rayType >= f->numRayTypes) return GRT_ERROR_INVALID_PARAMETER;
        t.funcTable = f->dEntries;
        t.numGeomTypes = f->numGeomTypes;
    }
    *out = t;
    return GRT_SUCCESS;
}

grtError grtTraceClosest(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, uint32_t rayCount,
                         grtHit* hits, grtFuncTable table, const grtTraceOptions* options, void* stream) {
    return launchTrace<false>(ctx, scene, geom, rays, rayCount, hits, table, options, stream);
}

grtError grtTraceAnyHit(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, uint32_t rayCount,
                        grtHit* hits, grtFuncTable table, const grtTraceOptions* options, void* stream) {
    return launchTrace<true>(ctx, scene, geom, rays, rayCount, hits, table, options, stream);
}

grtError grtTraceAllHits(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, uint32_t rayCount,
                         grtHit* hits, uint32_t maxHitsPerRay, uint32_t* hitCounts, grtFuncTable table,
                         const grtTraceOptions* options, void* stream) {
    if (!ctx || maxHitsPerRay == 0) return GRT_ERROR_INVALID_PARAMETER;
    if (rayCount && (!rays || !hits || !hitCounts || ((uintptr_t)rays & 15))) return GRT_ERROR_INVALID_PARAMETER;
    const BvhObject* g = geom ? findBvh(geom) : nullptr;
    if (g && g->split) return GRT_ERROR_INVALID_PARAMETER;  // a triangle would be met once per reference
    Context* c = asContext(ctx);
    TraceParams P{};
    bool isScene = false;
    int bs = 128;
    grtError e = prepareTrace(c, scene, geom, table, options, P, &isScene, &bs);
    if (e != GRT_SUCCESS || rayCount == 0) return e;
    P.rays = (const float4*)rays;
    P.hits = (uint32_t*)hits;
    P.count = rayCount;
    allHitsKernel<<<ceilDiv(rayCount, 128), 128, 0, (cudaStream_t)stream>>>(P, maxHitsPerRay, hitCounts);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    return GRT_SUCCESS;
}

grtError grtGenerateCameraRays(grtContext ctx, const grtCamera* camera, uint32_t width, uint32_t height, grtRay* rays,
                               void* stream) {
    if (!ctx || !camera || (width && height && !rays)) return GRT_ERROR_INVALID_PARAMETER;
    const size_t n = (size_t)width * height;
    if (n == 0) return GRT_SUCCESS;
    if (n > 0xFFFFFFFFull) return GRT_ERROR_INVALID_PARAMETER;
    cameraRayKernel<<<ceilDiv(n, 256), 256, 0, (cudaStream_t)stream>>>(*camera, width, height, (float4*)rays);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    return GRT_SUCCESS;
}

grtError grtGenerateUniformRays(grtContext ctx, const float lo[3], const float hi[3], uint64_t seed, uint32_t count,
                                float minT, float maxT, grtRay* rays, void* stream) {
    if (!ctx || !lo || !hi || (count && !rays) || ((uintptr_t)rays & 15)) return GRT_ERROR_INVALID_PARAMETER;
    for (int a = 0; a < 3; ++a)
        if (!(hi[a] >= lo[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a])) return GRT_ERROR_INVALID_PARAMETER;
    if (count == 0) return GRT_SUCCESS;
    const float3 l = make_float3(lo[0], lo[1], lo[2]);
    const float3 e = make_float3(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]);
    uniformRayKernel<<<ceilDiv(count, 256), 256, 0, (cudaStream_t)stream>>>(l, e, seed, count, minT, maxT,
                                                                               (float4*)rays);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    return GRT_SUCCESS;
}

static grtError sceneForShading(grtScene scene, BvhObject** out) {
    BvhObject* o = findBvh(scene);
    if (!o || o->primType != kPrimScene) return GRT_ERROR_INVALID_PARAMETER;
    if (!o->built) return GRT_ERROR_NOT_BUILT;
    *out = o;
    return GRT_SUCCESS;
}

grtError grtGenerateAORays(grtContext ctx, grtScene scene, const grtRay* primaryRays, const grtHit* primaryHits,
                           uint32_t pixelCount, uint32_t samplesPerPixel, uint64_t seed, float length, grtRay* aoRays,
                           void* stream) {
    if (!ctx || samplesPerPixel == 0) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = nullptr;
    grtError e = sceneForShading(scene, &o);
    if (e != GRT_SUCCESS || pixelCount == 0) return e;
    if (!primaryRays || !primaryHits || !aoRays) return GRT_ERROR_INVALID_PARAMETER;
    if ((size_t)pixelCount * samplesPerPixel > 0xFFFFFFFFull) return GRT_ERROR_INVALID_PARAMETER;
    aoRayKernel<<<ceilDiv(pixelCount, 128), 128, 0, (cudaStream_t)stream>>>(
        (const InstanceRecord*)o->leaves, o->primToLeaf, (const float4*)o->fwd32, (const float4*)primaryRays,
        (const uint32_t*)primaryHits, pixelCount, samplesPerPixel, seed, length, (float4*)aoRays);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    return GRT_SUCCESS;
}

grtError grtTraceAmbientOcclusion(grtContext ctx, grtScene scene, const grtRay* primaryRays, const grtHit* primaryHits,
                                  uint32_t pixelCount, uint32_t samplesPerPixel, uint64_t seed, float length, float* ao,
                                  const grtTraceOptions* options, void* stream) {
    if (!ctx || samplesPerPixel == 0) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    TraceParams P{};
    bool isScene = false;
    int bs = 128;
    grtError e = prepareTrace(c, scene, nullptr, nullptr, options, P, &isScene, &bs, 0.6f);
    if (e != GRT_SUCCESS || pixelCount == 0) return e;
    if (!primaryRays || !primaryHits || !ao) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = findBvh(scene);
    P.count = pixelCount;
    P.primaryRays = (const float4*)primaryRays;
    P.primaryHits = (const uint32_t*)primaryHits;
    P.sceneLeaves = (const InstanceRecord*)o->leaves;
    P.scenePrimToLeaf = o->primToLeaf;
    P.fwd32 = (const float4*)o->fwd32;
    P.spp = samplesPerPixel;
    P.seed = seed;
    P.aoLength = length;
    P.ao = ao;
    if ((size_t)pixelCount * samplesPerPixel > 0xFFFFFFFEull) return GRT_ERROR_INVALID_PARAMETER;
    const bool count = options && (options->flags & GRT_TRACE_FLAG_COUNT);
    void (*kernel)(TraceParams, const uint32_t*, const uint32_t*, uint32_t*, const float4*) =
        walkFormats(P, true) == kFmWide8 ? (count ? aoTraceKernel<true, kFmWide8> : aoTraceKernel<false, kFmWide8>)
        : walkFormats(P, true) == kFmQuant ? (count ? aoTraceKernel<true, kFmQuant> : aoTraceKernel<false, kFmQuant>)
                                           : (count ? aoTraceKernel<true> : aoTraceKernel<false>);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = (size_t)bs * traceSmemWords(P.sharedDepth, slotsOf(walkFormats(P, true))) * sizeof(uint32_t);
    LaunchShape L = persistentShape(c, kernel, bs, smem);
    // scratch after the global stack: the hit count (256 B), the list of hit pixels and
    // their AO frames (48 B each)
    void* extra = nullptr;
    const size_t listBytes = alignUp(4 * (size_t)pixelCount, 256);
    e = bindGlobalStack(c, options, L.blocks * bs, P, 256 + listBytes + 48 * (size_t)pixelCount, &extra);
    if (e != GRT_SUCCESS) return e;
    uint32_t* listCount = static_cast<uint32_t*>(extra);
    uint32_t* list = reinterpret_cast<uint32_t*>(static_cast<char*>(extra) + 256);
    float4* frames = reinterpret_cast<float4*>(static_cast<char*>(extra) + 256 + listBytes);
    uint32_t* counts = reinterpret_cast<uint32_t*>(ao);
    P.counter = nextCounter(c);
    GRT_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));
    GRT_CUDA(cudaMemsetAsync(listCount, 0, sizeof(uint32_t), s));
    aoCompactKernel<<<ceilDiv(pixelCount, 256), 256, 0, s>>>(P, pixelCount, list, listCount, counts, frames);
    kernel<<<L.blocks, bs, smem, s>>>(P, list, listCount, counts, frames);
    aoFinishKernel<<<smCount(c) * 4, 256, 0, s>>>(list, listCount, samplesPerPixel, ao);
    GRT_LAUNCH_CHECK();
    noteLaunches(3);
    return GRT_SUCCESS;
}

// ---------------------------------------------------------------- path tracing (Sec. 5)
// Path tracing with next event estimation as a wavefront over the library's own queries:
// per path vertex, closest hit of every live path ray, one shading pass, then any hit of
// the shadow rays that pass wrote. The shading pass (ptShadeKernel) first credits the
// previous vertex's light sample when its shadow ray found nothing, then:
//  * a miss adds T * sky and ends the path; a hit on an emitting triangle adds
//    T * emission at the first vertex only and ends the path;
//  * otherwise, in the hit's AO frame (face normal toward the ray, tangent v1 - v0,
//    origin p + 1e-4 n): one light triangle l = (xi_a * L) >> 24 in integers, a uniform
//    point q on it (s = sqrt(xi_b): (1-s) a + s (1-xi_c) b + s xi_c c), and if
//    cos_s > 0 and |cos_l| > 0 a shadow ray over [0, dist (1 - 1e-4)] with the pending
//    contribution T * (albedo / pi) * cos_s |cos_l| / dist^2 * emission_l * L * area_l;
//    the next ray leaves along a cosine-weighted direction (xi_d, xi_e); T *= albedo.
// Random numbers: xi(seed, ray, (sample * maxDepth + depth) * 3 + k, dim) with
// (k, dim) = (0,0) a, (0,1) b, (1,0) c, (1,1) d, (2,0) e.
struct PathParams {
    float4* pathRays;
    uint32_t* pathHits;
    float4* shadowRays;
    uint32_t* shadowHits;
    float4* T;        // throughput (xyz)
    float4* L;        // radiance of the current sample (xyz)
    float4* pending;  // light sample waiting for its shadow ray (xyz)
    const float* albedo;
    const float* emission;
    const uint32_t* materialOffset;
    const uint32_t* lights;
    uint32_t lightCount;
    uint32_t instanceCount;  // of the scene: light entries naming another instance are rejected
    uint32_t maxDepth;
    uint32_t n;
    uint32_t sample;
    uint32_t spp;
    uint64_t seed;
    float3 sky;
};

__device__ __forceinline__ uint32_t sampleBits24(uint64_t seed, uint64_t pixel, uint32_t sample, uint32_t dim) {
    const uint64_t c = (pixel << 32) | ((uint64_t)sample << 1) | dim;
    return (uint32_t)(mix64(seed + (c + 1ull) * 0x9E3779B97F4A7C15ull) >> 40);
}

__device__ __forceinline__ float3 loadColour(const float* f, size_t m) {
    return make_float3(__ldg(f + 3 * m), __ldg(f + 3 * m + 1), __ldg(f + 3 * m + 2));
}

// World-space vertices of primitive `prim` of instance `inst` (float32 forward frame).
__device__ __forceinline__ void worldTriangle(const TraceParams& P, uint32_t inst, uint32_t prim, float3 v[3]) {
    const InstanceRecord* R = P.sceneLeaves + P.scenePrimToLeaf[inst];
    const BvhHeader* g = R->geometry;
    const float4* rec = reinterpret_cast<const float4*>(g->leaves) + 3 * (size_t)g->primToLeaf[prim];
    const float4* fr = P.fwd32 + kFrameRows * (size_t)inst;
    const float4 m0 = fr[0], m1 = fr[1], m2 = fr[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float3 o = f3(rec[k]);
        v[k] = make_float3(m0.x * o.x + m0.y * o.y + m0.z * o.z + m0.w, m1.x * o.x + m1.y * o.y + m1.z * o.z + m1.w,
                           m2.x * o.x + m2.y * o.y + m2.z * o.z + m2.w);
    }
}

__global__ void __launch_bounds__(256) ptInitKernel(PathParams Q, const float4* rays) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Q.n) return;
    Q.pathRays[2 * (size_t)i] = rays[2 * (size_t)i];
    Q.pathRays[2 * (size_t)i + 1] = rays[2 * (size_t)i + 1];
    Q.T[i] = make_float4(1.f, 1.f, 1.f, 0.f);
    Q.L[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void creditPending(const PathParams& Q, uint32_t i) {
    if (Q.shadowRays[2 * (size_t)i + 1].w >= 0.f && Q.shadowHits[5 * (size_t)i + 1] == kInvalid) {
        const float4 c = Q.pending[i], l = Q.L[i];
        Q.L[i] = make_float4(l.x + c.x, l.y + c.y, l.z + c.z, 0.f);
    }
}

__device__ __forceinline__ void endPath(const PathParams& Q, uint32_t i) {
    Q.pathRays[2 * (size_t)i + 1].w = -1.f;
    Q.shadowRays[2 * (size_t)i + 1] = make_float4(0.f, 0.f, 0.f, -1.f);
}

__global__ void __launch_bounds__(256) ptShadeKernel(TraceParams P, PathParams Q, uint32_t depth) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Q.n) return;
    if (depth > 0) creditPending(Q, i);
    const float4* ray = Q.pathRays + 2 * (size_t)i;
    if (ray[1].w < 0.f) {  // the path has ended
        Q.shadowRays[2 * (size_t)i + 1] = make_float4(0.f, 0.f, 0.f, -1.f);
        return;
    }
    const uint32_t* hit = Q.pathHits + 5 * (size_t)i;
    const float4 T = Q.T[i];
    float4 L = Q.L[i];
    if (hit[1] == kInvalid) {
        Q.L[i] = make_float4(L.x + T.x * Q.sky.x, L.y + T.y * Q.sky.y, L.z + T.z * Q.sky.z, 0.f);
        endPath(Q, i);
        return;
    }
    const size_t m = (size_t)Q.materialOffset[hit[0]] + hit[1];
    const float3 Le = loadColour(Q.emission, m);
    if (Le.x != 0.f || Le.y != 0.f || Le.z != 0.f) {
        if (depth == 0) Q.L[i] = make_float4(L.x + T.x * Le.x, L.y + T.y * Le.y, L.z + T.z * Le.z, 0.f);
        endPath(Q, i);
        return;
    }
    AoFrame F;
    aoFrame(P.sceneLeaves, P.scenePrimToLeaf, P.fwd32, ray, hit, F);
    const float3 rho = loadColour(Q.albedo, m);
    const uint32_t j = (Q.sample * Q.maxDepth + depth) * 3u;
    float4 sray1 = make_float4(0.f, 0.f, 0.f, -1.f);
    if (Q.lightCount > 0) {
        const uint32_t ka = sampleBits24(Q.seed, i, j, 0);
        const uint32_t li = (uint32_t)(((uint64_t)ka * Q.lightCount) >> 24);
        const uint32_t linst = Q.lights[2 * (size_t)li], lprim = Q.lights[2 * (size_t)li + 1];
        bool lightOk = linst < Q.instanceCount;
        if (lightOk) {
            const InstanceRecord* R = P.sceneLeaves + P.scenePrimToLeaf[linst];
            lightOk = instPrimType(R->typeBits) == GRT_PRIMITIVE_TRIANGLE_MESH && lprim < R->geometry->primCount;
        }
        if (!lightOk) {
            latchError(P.error, GRT_ERROR_INVALID_PARAMETER);  // no light sample from a bad entry
        } else {
            float3 v[3];
            worldTriangle(P, linst, lprim, v);
            const float3 cr = cross3(v[1] - v[0], v[2] - v[0]);
            const float area2 = sqrtf(dot3(cr, cr));  // twice the area
            const float3 nl = cr * (1.0f / area2);
            const float su = sqrtf(sampleXi(Q.seed, i, j, 1)), xc = sampleXi(Q.seed, i, j + 1, 0);
            const float3 q = v[0] * (1.f - su) + v[1] * (su * (1.f - xc)) + v[2] * (su * xc);
            float3 w = q - F.org;
            const float dist = sqrtf(dot3(w, w));
            w = w * (1.0f / dist);
            const float cs = dot3(F.n, w), cl = fabsf(dot3(nl, w));
            if (cs > 0.f && cl > 0.f) {
                const float3 El = loadColour(Q.emission, (size_t)Q.materialOffset[linst] + lprim);
                const float k =
                    cs * cl / (dist * dist) * (float)Q.lightCount * (0.5f * area2) * (1.0f / 3.14159265358979f);
                Q.pending[i] = make_float4(T.x * rho.x * El.x * k, T.y * rho.y * El.y * k, T.z * rho.z * El.z * k, 0.f);
                Q.shadowRays[2 * (size_t)i] = make_float4(F.org.x, F.org.y, F.org.z, 0.f);
                sray1 = make_float4(w.x, w.y, w.z, dist * (1.f - 1e-4f));
            }
        }
    }
    Q.shadowRays[2 * (size_t)i + 1] = sray1;
    // next direction: cosine-weighted about n, the AO frame's sample form
    const float xd = sampleXi(Q.seed, i, j + 1, 1), xe = sampleXi(Q.seed, i, j + 2, 0);
    float sn, cs2;
    sincospif(2.0f * xd, &sn, &cs2);
    const float r = sqrtf(xe);
    const float3 dir = F.tg * (cs2 * r) + F.bt * (sn * r) + F.n * sqrtf(1.0f - xe);
    Q.T[i] = make_float4(T.x * rho.x, T.y * rho.y, T.z * rho.z, 0.f);
    Q.pathRays[2 * (size_t)i] = make_float4(F.org.x, F.org.y, F.org.z, 0.f);
    Q.pathRays[2 * (size_t)i + 1] = make_float4(dir.x, dir.y, dir.z, INFINITY);
}

__global__ void __launch_bounds__(256) ptFinishKernel(PathParams Q, float* radiance) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Q.n) return;
    creditPending(Q, i);
    const float4 l = Q.L[i];
    const float inv = 1.0f / (float)Q.spp;
    float* out = radiance + 3 * (size_t)i;
    if (Q.sample == 0) {
        out[0] = l.x * inv, out[1] = l.y * inv, out[2] = l.z * inv;
    } else {
        out[0] += l.x * inv, out[1] += l.y * inv, out[2] += l.z * inv;
    }
}

// Workspace of a path trace of n rays: path rays, path hits, shadow rays, shadow hits,
// throughput, radiance, pending light samples.
static size_t pathWorkspace(uint32_t n, size_t off[7]) {
    const size_t sizes[7] = {32 * (size_t)n, 20 * (size_t)n, 32 * (size_t)n, 20 * (size_t)n,
                             16 * (size_t)n, 16 * (size_t)n, 16 * (size_t)n};
    size_t at = 0;
    for (int k = 0; k < 7; ++k) {
        off[k] = at;
        at = alignUp(at + sizes[k], 256);
    }
    return at;
}

grtError grtGetPathTraceWorkspaceSize(uint32_t rayCount, size_t* sizeBytes) {
    if (!sizeBytes) return GRT_ERROR_INVALID_PARAMETER;
    size_t off[7];
    *sizeBytes = pathWorkspace(rayCount, off);
    return GRT_SUCCESS;
}

grtError grtPathTrace(grtContext ctx, grtScene scene, const grtRay* rays, uint32_t rayCount,
                      const grtPathTraceInput* input, void* workspace, float* radiance,
                      const grtTraceOptions* options, void* stream) {
    if (!ctx || !input || input->maxDepth == 0 || input->samplesPerPixel == 0) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    TraceParams P{};
    bool isScene = false;
    int bs = 128;
    grtError e = prepareTrace(c, scene, nullptr, nullptr, options, P, &isScene, &bs);
    if (e != GRT_SUCCESS || rayCount == 0) return e;
    if (!rays || !radiance || !workspace || ((uintptr_t)rays & 15) || ((uintptr_t)workspace & 255))
        return GRT_ERROR_INVALID_PARAMETER;
    if (!input->albedo || !input->emission || !input->materialOffset || (input->lightCount && !input->lights))
        return GRT_ERROR_INVALID_PARAMETER;
    if ((uint64_t)input->samplesPerPixel * input->maxDepth * 3 >= 0x80000000ull) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = findBvh(scene);
    P.sceneLeaves = (const InstanceRecord*)o->leaves;
    P.scenePrimToLeaf = o->primToLeaf;
    P.fwd32 = (const float4*)o->fwd32;
    size_t off[7];
    pathWorkspace(rayCount, off);
    char* w = static_cast<char*>(workspace);
    PathParams Q{};
    Q.pathRays = reinterpret_cast<float4*>(w + off[0]);
    Q.pathHits = reinterpret_cast<uint32_t*>(w + off[1]);
    Q.shadowRays = reinterpret_cast<float4*>(w + off[2]);
    Q.shadowHits = reinterpret_cast<uint32_t*>(w + off[3]);
    Q.T = reinterpret_cast<float4*>(w + off[4]);
    Q.L = reinterpret_cast<float4*>(w + off[5]);
    Q.pending = reinterpret_cast<float4*>(w + off[6]);
    Q.albedo = input->albedo;
    Q.emission = input->emission;
    Q.materialOffset = input->materialOffset;
    Q.lights = input->lights;
    Q.lightCount = input->lightCount;
    Q.instanceCount = o->primCount;
    Q.maxDepth = input->maxDepth;
    Q.n = rayCount;
    Q.spp = input->samplesPerPixel;
    Q.seed = input->seed;
    Q.sky = make_float3(input->sky[0], input->sky[1], input->sky[2]);
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = ceilDiv(rayCount, 256);
    for (uint32_t smp = 0; smp < Q.spp; ++smp) {
        Q.sample = smp;
        ptInitKernel<<<blocks, 256, 0, s>>>(Q, (const float4*)rays);
        GRT_LAUNCH_CHECK();
        noteLaunches(1);
        for (uint32_t depth = 0; depth < Q.maxDepth; ++depth) {
            e = launchTrace<false>(ctx, scene, nullptr, (const grtRay*)Q.pathRays, rayCount, (grtHit*)Q.pathHits,
                                   nullptr, options, stream);
            if (e != GRT_SUCCESS) return e;
            ptShadeKernel<<<blocks, 256, 0, s>>>(P, Q, depth);
            GRT_LAUNCH_CHECK();
            noteLaunches(1);
            e = launchTrace<true>(ctx, scene, nullptr, (const grtRay*)Q.shadowRays, rayCount, (grtHit*)Q.shadowHits,
                                  nullptr, options, stream);
            if (e != GRT_SUCCESS) return e;
        }
        ptFinishKernel<<<blocks, 256, 0, s>>>(Q, radiance);
        GRT_LAUNCH_CHECK();
        noteLaunches(1);
    }
    return GRT_SUCCESS;
}

// Shared-memory budget of the adjoint's block-private gradient copy (4,096 vertices).
static constexpr size_t kShadePrivateBytes = 96 * 1024;

// The shading parameters of one call: the target (a triangle geometry, or a scene with
// per-instance triangle offsets into the mesh arrays) and the mesh arrays.
static grtError prepareShade(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, uint32_t n,
                             const uint32_t* triOffset, const uint32_t* indices, const float* positions,
                             const float* colours, const float* light, const grtTraceOptions* options, TraceParams& P,
                             ShadeParams& S, int* bs) {
    if (!ctx || (scene != nullptr) == (geom != nullptr)) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = findBvh(scene ? (const void*)scene : (const void*)geom);
    if (!o) return GRT_ERROR_INVALID_PARAMETER;
    if (geom && o->primType != GRT_PRIMITIVE_TRIANGLE_MESH) return GRT_ERROR_INVALID_PARAMETER;
    bool isScene = false;
    grtError e = prepareTrace(asContext(ctx), scene, geom, nullptr, options, P, &isScene, bs);
    if (e != GRT_SUCCESS) return e;
    if (n && (!rays || !indices || !positions || !colours || !light || ((uintptr_t)rays & 15)))
        return GRT_ERROR_INVALID_PARAMETER;
    if (n && scene && !triOffset) return GRT_ERROR_INVALID_PARAMETER;
    S.rays = (const float4*)rays;
    S.n = n;
    S.idx = indices;
    S.pos = positions;
    S.col = colours;
    S.light = light;
    if (scene) {
        S.triOffset = triOffset;
        S.frames = (const float4*)o->fwd32;
        S.sceneLeaves = (const InstanceRecord*)o->leaves;
        S.scenePrimToLeaf = o->primToLeaf;
    }
    return GRT_SUCCESS;
}

// The forward shading launch (image and / or visibility from stored hits).
static grtError launchShadeForward(Context* c, bool scene, TraceParams& P, const ShadeParams& S, int bs,
                                   const grtTraceOptions* options, cudaStream_t s) {
    void (*kernel)(TraceParams, ShadeParams) =
        walkFormats(P, scene) == kFmWide8
            ? (scene ? shadeForwardKernel<true, kFmWide8> : shadeForwardKernel<false, kFmWide8>)
        : walkFormats(P, scene) == kFmQuant
            ? (scene ? shadeForwardKernel<true, kFmQuant> : shadeForwardKernel<false, kFmQuant>)
            : (scene ? shadeForwardKernel<true> : shadeForwardKernel<false>);
    const size_t smem = (size_t)bs * traceSmemWords(P.sharedDepth, slotsOf(walkFormats(P, scene))) * sizeof(uint32_t);
    LaunchShape L = persistentShape(c, kernel, bs, smem);
    L.blocks = std::min<int>(L.blocks, (int)ceilDiv(S.n, bs));
    grtError e = bindGlobalStack(c, options, L.blocks * bs, P);
    if (e != GRT_SUCCESS) return e;
    P.counter = nextCounter(c);
    GRT_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));
    kernel<<<L.blocks, bs, smem, s>>>(P, S);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    return GRT_SUCCESS;
}

// The adjoint. Without stored hits (hits = NULL) it first traces them again with the
// library's closest-hit query and the forward's visibility pass, into context memory
// that lives only for this call, then runs the stored-hit adjoint over them: the
// recompute costs about one forward pass.
static grtError shadeBackward(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, const grtHit* hits,
                              const uint8_t* visibility, uint32_t n, const uint32_t* triOffset,
                              const uint32_t* indices, const float* positions, uint32_t nv, const float* colours,
                              const float* light, const float* gradImage, float* gradColours, float* gradLight,
                              float* gradPositions, const grtTraceOptions* options, void* stream) {
    TraceParams P{};
    ShadeParams S{};
    int bs = 128;
    grtError e = prepareShade(ctx, scene, geom, rays, n, triOffset, indices, positions, colours, light, options, P,
                              S, &bs);
    if (e != GRT_SUCCESS || n == 0) return e;
    if (!gradImage || !gradColours || !gradLight || !gradPositions) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    if (!hits) {
        void* aux = nullptr;
        const size_t hitBytes = alignUp((size_t)n * sizeof(grtHit), 256);
        e = contextAux(c, hitBytes + n, &aux);
        if (e != GRT_SUCCESS) return e;
        grtHit* th = (grtHit*)aux;
        uint8_t* tv = (uint8_t*)aux + hitBytes;
        e = launchTrace<false>(ctx, scene, geom, rays, n, th, nullptr, options, stream);
        if (e != GRT_SUCCESS) return e;
        TraceParams Pv = P;
        ShadeParams Sv = S;
        Sv.hits = (const uint32_t*)th;
        Sv.image = nullptr;
        Sv.vis = tv;
        e = launchShadeForward(c, scene != nullptr, Pv, Sv, bs, options, s);
        if (e != GRT_SUCCESS) return e;
        hits = th;
        visibility = tv;
    }
    S.hits = (const uint32_t*)hits;
    S.vis = const_cast<uint8_t*>(visibility);
    S.gimg = gradImage;
    S.gcol = gradColours;
    S.glight = gradLight;
    S.gpos = gradPositions;
    // block-private gradient copy when the mesh's vertex count is known and its 24 bytes
    // per vertex fit the budget
    const bool priv = nv > 0 && (size_t)nv * 24 <= kShadePrivateBytes;
    void (*kernel)(TraceParams, ShadeParams, uint32_t) =
        scene ? (priv ? shadeBackwardKernel<true, true> : shadeBackwardKernel<true, false>)
              : (priv ? shadeBackwardKernel<false, true> : shadeBackwardKernel<false, false>);
    const size_t smem = priv ? (size_t)nv * 24 : 0;
    if (smem > 48 * 1024) GRT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LaunchShape L = persistentShape(c, kernel, bs, smem);
    // the adjoint traces nothing: 8 blocks per SM keep each block's share of pixels large
    // next to its pass over the private copy
    L.blocks = std::min(L.blocks, 8 * smCount(c));
    L.blocks = std::min<int>(L.blocks, (int)ceilDiv(n, bs));
    P.counter = nextCounter(c);
    GRT_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));
    kernel<<<L.blocks, bs, smem, s>>>(P, S, priv ? nv : 0u);
    GRT_LAUNCH_CHECK();
    noteLaunches(1);
    return GRT_SUCCESS;
}

static grtError shadeForward(grtContext ctx, grtScene scene, grtGeometry geom, const grtRay* rays, const grtHit* hits,
                             uint32_t n, const uint32_t* triOffset, const uint32_t* indices, const float* positions,
                             const float* colours, const float* light, float* image, uint8_t* visibility,
                             const grtTraceOptions* options, void* stream) {
    TraceParams P{};
    ShadeParams S{};
    int bs = 128;
    grtError e = prepareShade(ctx, scene, geom, rays, n, triOffset, indices, positions, colours, light, options, P,
                              S, &bs);
    if (e != GRT_SUCCESS || n == 0) return e;
    if (!hits || !image) return GRT_ERROR_INVALID_PARAMETER;
    S.hits = (const uint32_t*)hits;
    S.image = image;
    S.vis = visibility;
    return launchShadeForward(asContext(ctx), scene != nullptr, P, S, bs, options, (cudaStream_t)stream);
}

grtError grtShadeLambert(grtContext ctx, grtGeometry geom, const grtRay* rays, const grtHit* hits, uint32_t pixelCount,
                         const uint32_t* indices, const float* positions, const float* colours, const float* light,
                         float* image, uint8_t* visibility, const grtTraceOptions* options, void* stream) {
    if (!geom) return GRT_ERROR_INVALID_PARAMETER;
    return shadeForward(ctx, nullptr, geom, rays, hits, pixelCount, nullptr, indices, positions, colours, light, image,
                        visibility, options, stream);
}

grtError grtShadeLambertBackward(grtContext ctx, grtGeometry geom, const grtRay* rays, const grtHit* hits,
                                 const uint8_t* visibility, uint32_t pixelCount, const uint32_t* indices,
                                 const float* positions, const float* colours, const float* light,
                                 const float* gradImage, float* gradColours, float* gradLight, float* gradPositions,
                                 const grtTraceOptions* options, void* stream) {
    BvhObject* o = geom ? findBvh(geom) : nullptr;
    if (!o) return GRT_ERROR_INVALID_PARAMETER;
    return shadeBackward(ctx, nullptr, geom, rays, hits, visibility, pixelCount, nullptr, indices, positions,
                         o->vertexCount, colours, light, gradImage, gradColours, gradLight, gradPositions, options,
                         stream);
}

grtError grtShadeLambertScene(grtContext ctx, grtScene scene, const grtRay* rays, const grtHit* hits,
                              uint32_t pixelCount, const uint32_t* instanceTriangleOffset, const uint32_t* indices,
                              const float* positions, const float* colours, const float* light, float* image,
                              uint8_t* visibility, const grtTraceOptions* options, void* stream) {
    if (!scene) return GRT_ERROR_INVALID_PARAMETER;
    return shadeForward(ctx, scene, nullptr, rays, hits, pixelCount, instanceTriangleOffset, indices, positions,
                        colours, light, image, visibility, options, stream);
}

grtError grtShadeLambertSceneBackward(grtContext ctx, grtScene scene, const grtRay* rays, const grtHit* hits,
                                      const uint8_t* visibility, uint32_t pixelCount,
                                      const uint32_t* instanceTriangleOffset, const uint32_t* indices,
                                      const float* positions, uint32_t vertexCount, const float* colours,
                                      const float* light, const float* gradImage, float* gradColours, float* gradLight,
                                      float* gradPositions, const grtTraceOptions* options, void* stream) {
    if (!scene) return GRT_ERROR_INVALID_PARAMETER;
    return shadeBackward(ctx, scene, nullptr, rays, hits, visibility, pixelCount, instanceTriangleOffset, indices,
                         positions, vertexCount, colours, light, gradImage, gradColours, gradLight, gradPositions,
                         options, stream);
}

}  // extern "C"
