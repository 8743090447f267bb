// A user kernel that traces rays itself through grt_device.cuh: one ray per thread,
// closest or any hit, hit records written like the library's own queries.
#include <cuda_runtime.h>

#include "grt_device.cuh"

__global__ void userTrace(grtDeviceTarget T, const float4* rays, uint32_t n, grtHit* hits, int anyHit) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = rays[2 * (size_t)i], b = rays[2 * (size_t)i + 1];
    const float3 o = make_float3(a.x, a.y, a.z), d = make_float3(b.x, b.y, b.z);
    hits[i] = anyHit ? grt_device::traceAnyHit(T, o, d, a.w, b.w) : grt_device::traceClosest(T, o, d, a.w, b.w);
}

extern "C" int userTraceLaunch(const grtDeviceTarget* T, const void* rays, uint32_t n, void* hits, int anyHit,
                               void* stream) {
    if (n == 0) return 0;
    userTrace<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*T, (const float4*)rays, n, (grtHit*)hits, anyHit);
    return (int)cudaGetLastError();
}
