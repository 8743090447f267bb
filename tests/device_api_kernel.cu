// A user kernel that traces rays itself through grt_device.cuh: one ray per thread,
// closest or any hit (optionally under a ray mask), hit records written like the
// library's own queries.
#include <cuda_runtime.h>

#include "grt_device.cuh"

__global__ void userTrace(grtDeviceTarget T, const float4* rays, uint32_t n, grtHit* hits, int anyHit,
                          uint32_t rayMask) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = rays[2 * (size_t)i], b = rays[2 * (size_t)i + 1];
    const float3 o = make_float3(a.x, a.y, a.z), d = make_float3(b.x, b.y, b.z);
    hits[i] = anyHit ? grt_device::traceAnyHit(T, o, d, a.w, b.w, rayMask)
                     : grt_device::traceClosest(T, o, d, a.w, b.w, rayMask);
}

extern "C" int userTraceLaunch(const grtDeviceTarget* T, const void* rays, uint32_t n, void* hits, int anyHit,
                               void* stream) {
    if (n == 0) return 0;
    userTrace<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*T, (const float4*)rays, n, (grtHit*)hits, anyHit,
                                                                0xFFFFFFFFu);
    return (int)cudaGetLastError();
}

extern "C" int userTraceMaskedLaunch(const grtDeviceTarget* T, const void* rays, uint32_t n, void* hits, int anyHit,
                                     uint32_t rayMask, void* stream) {
    if (n == 0) return 0;
    userTrace<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*T, (const float4*)rays, n, (grtHit*)hits, anyHit,
                                                                rayMask);
    return (int)cudaGetLastError();
}

// Every hit of each ray through grt_device::AllHits: the first maxHits stored, the rest
// of the slots set to misses, the total count written.
__global__ void userAllHits(grtDeviceTarget T, const float4* rays, uint32_t n, grtHit* hits, uint32_t maxHits,
                            uint32_t* counts) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = rays[2 * (size_t)i], b = rays[2 * (size_t)i + 1];
    grt_device::AllHits<96> w(T, make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z), a.w, b.w);
    uint32_t k = 0;
    for (grtHit h = w.getNextHit(); h.primID != 0xFFFFFFFFu; h = w.getNextHit()) {
        if (k < maxHits) hits[(size_t)i * maxHits + k] = h;
        ++k;
    }
    grtHit miss;
    miss.instanceID = miss.primID = 0xFFFFFFFFu;
    miss.t = __int_as_float(0x7f800000);
    miss.u = miss.v = 0.f;
    for (uint32_t j = k; j < maxHits; ++j) hits[(size_t)i * maxHits + j] = miss;
    counts[i] = w.done() ? k : 0xFFFFFFFFu;
}

extern "C" int userAllHitsLaunch(const grtDeviceTarget* T, const void* rays, uint32_t n, void* hits, uint32_t maxHits,
                                 void* counts, void* stream) {
    if (n == 0) return 0;
    userAllHits<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*T, (const float4*)rays, n, (grtHit*)hits, maxHits,
                                                                   (uint32_t*)counts);
    return (int)cudaGetLastError();
}

// User intersection code (Sec. 7.4): discs stored as two float4 per primitive, {centre,
// radius} and {unit normal, 0}; the plane hit inside the radius (rim included) in
// [minT, maxT]. The payload counts this ray's intersector calls. A user filter (Sec.
// 7.6) that keeps hits on even primitive IDs only.
struct DiscFunctions {
    __device__ bool intersect(uint32_t func, const grtRay& r, const void* data, void* payload, grtHit& hit) const {
        if (func != GRT_INTERSECT_USER) return false;
        if (payload) ++*static_cast<uint32_t*>(payload);
        const float4* D = static_cast<const float4*>(data) + 2 * (size_t)hit.primID;
        const float4 a = D[0], b = D[1];
        const float den = r.direction[0] * b.x + r.direction[1] * b.y + r.direction[2] * b.z;
        if (den == 0.f) return false;
        const float t = ((a.x - r.origin[0]) * b.x + (a.y - r.origin[1]) * b.y + (a.z - r.origin[2]) * b.z) / den;
        if (!(t >= r.minT && t <= r.maxT)) return false;
        const float px = r.origin[0] + t * r.direction[0] - a.x, py = r.origin[1] + t * r.direction[1] - a.y,
                    pz = r.origin[2] + t * r.direction[2] - a.z;
        if (px * px + py * py + pz * pz > a.w * a.w) return false;
        hit.t = t;
        hit.u = hit.v = 0.f;
        return true;
    }
    __device__ bool filter(uint32_t func, const grtRay&, const void*, void*, const grtHit& hit) const {
        return func != GRT_FILTER_USER || (hit.primID & 1u) == 0;
    }
};

__global__ void userTraceDiscs(grtDeviceTarget T, const float4* rays, uint32_t n, grtHit* hits, int anyHit,
                               uint32_t* calls) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = rays[2 * (size_t)i], b = rays[2 * (size_t)i + 1];
    const float3 o = make_float3(a.x, a.y, a.z), d = make_float3(b.x, b.y, b.z);
    uint32_t c = 0;
    const DiscFunctions fn;
    hits[i] = anyHit ? grt_device::traceAnyHit(T, o, d, a.w, b.w, 0xFFFFFFFFu, fn, &c)
                     : grt_device::traceClosest(T, o, d, a.w, b.w, 0xFFFFFFFFu, fn, &c);
    calls[i] = c;
}

extern "C" int userTraceDiscsLaunch(const grtDeviceTarget* T, const void* rays, uint32_t n, void* hits, int anyHit,
                                    void* calls, void* stream) {
    if (n == 0) return 0;
    userTraceDiscs<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*T, (const float4*)rays, n, (grtHit*)hits,
                                                                     anyHit, (uint32_t*)calls);
    return (int)cudaGetLastError();
}

// Every hit through the disc functions (AllHits with a functor).
__global__ void userAllHitsDiscs(grtDeviceTarget T, const float4* rays, uint32_t n, grtHit* hits, uint32_t maxHits,
                                 uint32_t* counts) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = rays[2 * (size_t)i], b = rays[2 * (size_t)i + 1];
    grt_device::AllHits<96, DiscFunctions> w(T, make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z), a.w, b.w,
                                             0xFFFFFFFFu, DiscFunctions{});
    uint32_t k = 0;
    for (grtHit h = w.getNextHit(); h.primID != 0xFFFFFFFFu; h = w.getNextHit()) {
        if (k < maxHits) hits[(size_t)i * maxHits + k] = h;
        ++k;
    }
    grtHit miss;
    miss.instanceID = miss.primID = 0xFFFFFFFFu;
    miss.t = __int_as_float(0x7f800000);
    miss.u = miss.v = 0.f;
    for (uint32_t j = k; j < maxHits; ++j) hits[(size_t)i * maxHits + j] = miss;
    counts[i] = k;
}

extern "C" int userAllHitsDiscsLaunch(const grtDeviceTarget* T, const void* rays, uint32_t n, void* hits,
                                      uint32_t maxHits, void* counts, void* stream) {
    if (n == 0) return 0;
    userAllHitsDiscs<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*T, (const float4*)rays, n, (grtHit*)hits,
                                                                       maxHits, (uint32_t*)counts);
    return (int)cudaGetLastError();
}
