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
