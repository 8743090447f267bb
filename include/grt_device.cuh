/*
 * grt_device.cuh - ray queries from user CUDA kernels (sm_103a).
 *
 * The paper's device-side traversal object (Sec. 7.5) traces one ray from inside a
 * user's own kernel against a geometry or a scene and returns its hit record. Here a
 * host call, grtGetDeviceTarget (grt.h), describes the built geometry or scene (and an
 * optional function table) as a plain struct; the kernel passes it by value to
 *
 *   grtHit grt_device::traceClosest<DEPTH>(target, origin, direction, minT, maxT)
 *   grtHit grt_device::traceAnyHit<DEPTH>(target, origin, direction, minT, maxT)
 *   grt_device::AllHits<DEPTH>(target, origin, direction, minT, maxT).getNextHit()
 *
 * which run the library's own traversal (the same certified float32 tests with their
 * FP64 fallback; closest hits get t, u, v recomputed in FP64) on a per-thread stack of
 * DEPTH entries in local memory. A ray needing more entries stops early and latches
 * GRT_ERROR_STACK_OVERFLOW in the context's error word. The records follow grtHit:
 * a miss has primID = instanceID = 0xFFFFFFFF and t = +inf.
 *
 * The traversal code is compiled into the user's kernel: compile with
 *   nvcc -gencode arch=compute_103a,code=sm_103a -I <repo>/include -I <package>/csrc
 * (the package's csrc directory holds traverse.cuh). No device symbol of libgrt.so is
 * needed; the host side links libgrt.so for grtGetDeviceTarget only.
 */
#pragma once

#include "grt.h"
#include "traverse.cuh"

namespace grt_device {

namespace detail {

__device__ __forceinline__ grt::TraceParams params(const grtDeviceTarget& T, uint32_t rayMask) {
    grt::TraceParams P{};
    P.rayMask = rayMask ? rayMask : 0xFFFFFFFFu;
    P.target.nodes = static_cast<const float4*>(T.nodes);
    P.target.leaves = T.leaves;
    P.target.primType = T.primType;
    P.target.geomType = T.geomType;
    P.target.empty = T.primCount == 0;
    P.table = static_cast<const grt::FuncEntry*>(T.funcTable);
    P.numGeomTypes = T.numGeomTypes;
    P.rayType = T.rayType;
    P.error = T.deviceError;
    P.maxSteps = 1u << 26;
    P.inv64 = static_cast<const grt::InstanceFrames64*>(T.frames64);
    P.fwd32 = static_cast<const float4*>(T.frames32);
    if (T.primType == grt::kPrimScene) {
        P.sceneLeaves = static_cast<const grt::InstanceRecord*>(T.leaves);
        P.scenePrimToLeaf = T.primToLeaf;
    } else {
        P.targetPrimToLeaf = T.primToLeaf;
    }
    return P;
}

template <bool ANY, int DEPTH>
__device__ __forceinline__ grtHit trace(const grtDeviceTarget& T, float3 o, float3 d, float tmin, float tmax,
                                        uint32_t rayMask) {
    const grt::TraceParams P = params(T, rayMask);
    uint32_t entries[DEPTH];
    grt::Stack st{nullptr, entries, 0u, (uint32_t)DEPTH, 1u, 0u};
    grt::Hit h = T.primType == grt::kPrimScene ? grt::traceRay<ANY, true>(P, st, o, d, tmin, tmax)
                                               : grt::traceRay<ANY, false>(P, st, o, d, tmin, tmax);
    if (!ANY) grt::refineOne(P, o, d, tmin, tmax, h);
    grtHit r;
    r.instanceID = h.inst;
    r.primID = h.prim;
    r.t = h.t;
    r.u = h.u;
    r.v = h.v;
    return r;
}

}  // namespace detail

// Closest hit of the ray o + t d, t in [tmin, tmax]. rayMask: instances whose mask
// shares no bit with it are skipped (0 = all bits set).
template <int DEPTH = 64>
__device__ __forceinline__ grtHit traceClosest(const grtDeviceTarget& T, float3 o, float3 d, float tmin, float tmax,
                                               uint32_t rayMask = 0xFFFFFFFFu) {
    return detail::trace<false, DEPTH>(T, o, d, tmin, tmax, rayMask);
}

// Some hit of the ray in [tmin, tmax] (the first found), or a miss.
template <int DEPTH = 64>
__device__ __forceinline__ grtHit traceAnyHit(const grtDeviceTarget& T, float3 o, float3 d, float tmin, float tmax,
                                              uint32_t rayMask = 0xFFFFFFFFu) {
    return detail::trace<true, DEPTH>(T, o, d, tmin, tmax, rayMask);
}

// Every hit of one ray (Sec. 7.5's all-hits use of the any-hit traversal object):
//   grt_device::AllHits<> w(target, o, d, tmin, tmax);
//   for (grtHit h = w.getNextHit(); h.primID != 0xFFFFFFFF; h = w.getNextHit()) ...
// Each (instance, primitive) whose intersection lies in [tmin, tmax] comes once, in
// traversal order (not sorted by t), with t, u, v recomputed in FP64; then a miss
// record. done() tells whether the walk is over (the paper's getCurrentState()). The
// object holds its own stack of DEPTH entries: construct it where it is used; do not
// copy it.
template <int DEPTH = 64>
class AllHits {
  public:
    __device__ AllHits(const grtDeviceTarget& T, float3 o, float3 d, float tmin, float tmax,
                       uint32_t rayMask = 0xFFFFFFFFu)
        : P_(detail::params(T, rayMask)) {
        walk_.begin(P_, o, d, tmin, tmax);
    }
    AllHits(const AllHits&) = delete;
    AllHits& operator=(const AllHits&) = delete;
    __device__ grtHit getNextHit() {
        const grt::Hit h = walk_.next(P_);
        grtHit r;
        r.instanceID = h.inst;
        r.primID = h.prim;
        r.t = h.t;
        r.u = h.u;
        r.v = h.v;
        return r;
    }
    __device__ bool done() const { return walk_.done(); }

  private:
    grt::TraceParams P_;
    grt::AllHitsWalk<DEPTH> walk_;
};

}  // namespace grt_device
