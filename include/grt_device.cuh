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
 * FP64 fallback; closest hits get t, u, v recomputed in double-float) on a per-thread stack of
 * DEPTH entries in local memory. A ray needing more entries stops early and latches
 * GRT_ERROR_STACK_OVERFLOW in the context's error word. The records follow grtHit:
 * a miss has primID = instanceID = 0xFFFFFFFF and t = +inf.
 *
 * User intersection and filter code (Sec. 7.4, 7.6) is a functor passed to these
 * calls (after the ray mask), with members
 *
 *   __device__ bool intersect(uint32_t func, const grtRay& ray, const void* data, void* payload,
 *                             grtHit& hit) const;
 *   __device__ bool filter(uint32_t func, const grtRay& ray, const void* data, void* payload,
 *                          const grtHit& hit) const;
 *
 * intersect is called for a custom primitive whose function-table entry names an ID
 * func >= GRT_INTERSECT_USER: hit.primID and hit.instanceID are set, data is the
 * entry's intersectFuncData, payload is what the caller passed. It returns true and
 * sets hit.t (and u, v) for an intersection in [ray.minT, ray.maxT]. The ray is in the
 * primitive's object space, with t measured along it as given (its origin may be
 * moved along the line; the library converts t back). filter is called for every hit
 * (triangles, built-in and user primitives) whose entry names a filter ID >=
 * GRT_FILTER_USER, with hit.t on the same ray; returning false rejects the hit and
 * traversal goes on. User functions get no FP64 fallback and their hits no FP64
 * refinement: their float32 arithmetic is the user's. The functor is inlined into the
 * traversal (no relocatable device code, no function pointers).
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
    P.target.fmt = T.nodeFormat & 0xFFu;
    P.target.split = (T.nodeFormat >> 8) & 1u;
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

template <bool ANY, int DEPTH, class Fn>
__device__ __forceinline__ grtHit trace(const grtDeviceTarget& T, float3 o, float3 d, float tmin, float tmax,
                                        uint32_t rayMask, const Fn* fn, void* payload) {
    const grt::TraceParams P = params(T, rayMask);
    uint32_t entries[DEPTH];
    grt::Stack st{nullptr, entries, 0u, (uint32_t)DEPTH, 1u, 0u};
    grt::Hit h = T.primType == grt::kPrimScene
                     ? grt::traceRay<ANY, true, false, Fn>(P, st, o, d, tmin, tmax, nullptr, fn, payload)
                     : grt::traceRay<ANY, false, false, Fn>(P, st, o, d, tmin, tmax, nullptr, fn, payload);
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

// The functor type of calls without user functions.
using NoCustom = grt::NoUser;

// Closest hit of the ray o + t d, t in [tmin, tmax]. rayMask: instances whose mask
// shares no bit with it are skipped (0 = all bits set). fn: user intersection / filter
// code (see above), payload: handed to it.
template <int DEPTH = 64, class Fn = NoCustom>
__device__ __forceinline__ grtHit traceClosest(const grtDeviceTarget& T, float3 o, float3 d, float tmin, float tmax,
                                               uint32_t rayMask = 0xFFFFFFFFu, const Fn& fn = Fn{},
                                               void* payload = nullptr) {
    return detail::trace<false, DEPTH, Fn>(T, o, d, tmin, tmax, rayMask, &fn, payload);
}

// Some hit of the ray in [tmin, tmax] (the first found), or a miss.
template <int DEPTH = 64, class Fn = NoCustom>
__device__ __forceinline__ grtHit traceAnyHit(const grtDeviceTarget& T, float3 o, float3 d, float tmin, float tmax,
                                              uint32_t rayMask = 0xFFFFFFFFu, const Fn& fn = Fn{},
                                              void* payload = nullptr) {
    return detail::trace<true, DEPTH, Fn>(T, o, d, tmin, tmax, rayMask, &fn, payload);
}

// Every hit of one ray (Sec. 7.5's all-hits use of the any-hit traversal object):
//   grt_device::AllHits<> w(target, o, d, tmin, tmax);
//   for (grtHit h = w.getNextHit(); h.primID != 0xFFFFFFFF; h = w.getNextHit()) ...
// Each (instance, primitive) whose intersection lies in [tmin, tmax] comes once, in
// traversal order (not sorted by t), with t, u, v recomputed in double-float; then a miss
// record. done() tells whether the walk is over (the paper's getCurrentState()). The
// object holds its own stack of DEPTH entries: construct it where it is used; do not
// copy it. With user functions: AllHits<DEPTH, Fn> w(target, o, d, tmin, tmax, mask, fn,
// payload) (the object keeps a copy of fn).
template <int DEPTH = 64, class Fn = NoCustom>
class AllHits {
  public:
    __device__ AllHits(const grtDeviceTarget& T, float3 o, float3 d, float tmin, float tmax,
                       uint32_t rayMask = 0xFFFFFFFFu, const Fn& fn = Fn{}, void* payload = nullptr)
        : P_(detail::params(T, rayMask)), fn_(fn) {
        walk_.user = &fn_;
        walk_.payload = payload;
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
    Fn fn_;
    grt::AllHitsWalk<DEPTH, Fn> walk_;
};

}  // namespace grt_device
