// Ray-query kernels (closest hit, any hit, fused ambient occlusion), ray generation
// (camera, ambient occlusion) and their host entry points. The traversal itself is in
// traverse.cuh.
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "traverse.cuh"

namespace grt {

// Persistent refill loop shared by the query kernels (warp-level ray compaction):
// each lane owns one work item and advances its ray one traversal step per iteration;
// when the warp's live lanes drop to P.refillBelow or fewer, the idle lanes take fresh
// items from the global queue with one atomic per warp, so short rays do not leave
// lanes idle while long ones finish. Src supplies the items:
//   count()             number of items (may be read from device memory)
//   begin(i, P, st, s)  set up item i's ray in s; false if the item has no ray
//   finish(i, s)        consume item i's result s.best
template <bool ANY, bool SCENE, bool COUNT, class Src>
__device__ __forceinline__ void refillLoop(const TraceParams& P, Stack& st, Src& src) {
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
        if (item != kNone && stepRay<ANY, SCENE, COUNT>(P, st, s, &v)) {
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

template <bool ANY, bool SCENE, bool COUNT>
__global__ void traceKernel(TraceParams P) {
    extern __shared__ uint32_t sstack[];
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    Stack st{sstack + threadIdx.x, P.globalStack + gtid, P.sharedDepth, P.globalDepth, P.globalStride, 0};
    RayBufferSource<SCENE> src{P.count, &P};
    refillLoop<ANY, SCENE, COUNT>(P, st, src);
}

// The closest hits' t, u, v recomputed in FP64, one thread per ray after traversal so
// that every lane of a warp takes part (FP64 is far slower than FP32 on this GPU).
__global__ void __launch_bounds__(256) refineKernel(TraceParams P) {
    const bool scene = P.target.primType == kPrimScene;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < P.count; r += gridDim.x * blockDim.x) {
        uint32_t* h = P.hits + 5 * (size_t)r;
        const uint32_t inst = h[0], prim = h[1];
        if (prim == kInvalid) continue;
        uint32_t primType, geomType;
        const void* leaves;
        const uint32_t* toLeaf;
        if (scene) {
            const InstanceRecord* R = P.sceneLeaves + P.scenePrimToLeaf[inst];
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
            rec = reinterpret_cast<const float4*>(leaves) + 3 * (size_t)toLeaf[prim];
        } else if (P.table && geomType < P.numGeomTypes) {
            const FuncEntry fe = P.table[(size_t)P.rayType * P.numGeomTypes + geomType];
            if (fe.func == GRT_INTERSECT_SPHERE) {
                rec = reinterpret_cast<const float4*>(fe.data) + prim;
                sphere = true;
            }
        }
        if (!rec) continue;
        const float4 a = P.rays[2 * (size_t)r], b = P.rays[2 * (size_t)r + 1];
        const float4 res = refine64(P.inv64, scene, inst, f3(a), f3(b), rec, sphere, a.w, b.w);
        if (res.w != 0.f) {
            h[2] = __float_as_uint(res.x);
            h[3] = __float_as_uint(res.y);
            h[4] = __float_as_uint(res.z);
        }
    }
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
//     per warp); every pixel's occlusion count starts at 0 (kept in ao's words);
//  2. aoTraceKernel: the refill loop over the list's (pixel, sample) items; each
//     item's ray is generated in registers and traced as an any-hit query, and an
//     occluded sample adds 1 to its pixel's count;
//  3. aoFinishKernel: ao = count / samplesPerPixel for the listed pixels.
__global__ void aoCompactKernel(const uint32_t* __restrict__ hits, uint32_t pixels, uint32_t* __restrict__ list,
                                uint32_t* __restrict__ listCount, uint32_t* __restrict__ counts) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool hit = p < pixels && hits[5 * (size_t)p + 1] != kInvalid;
    if (p < pixels) counts[p] = 0u;
    const uint32_t mask = __ballot_sync(0xffffffffu, hit);
    const uint32_t lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0 && mask) base = atomicAdd(listCount, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (hit) list[base + __popc(mask & ((1u << lane) - 1u))] = p;
}

struct AoSource {
    const TraceParams* P;
    const uint32_t* list;
    const uint32_t* listCount;
    uint32_t* counts;
    __device__ unsigned long long count() const { return (unsigned long long)*listCount * P->spp; }
    __device__ bool begin(uint32_t i, const TraceParams& Pm, Stack& st, RayState& s) const {
        const uint32_t slot = i / Pm.spp, smp = i - slot * Pm.spp;
        const uint32_t p = list[slot];
        AoFrame F;
        if (!aoFrame(Pm.sceneLeaves, Pm.scenePrimToLeaf, Pm.fwd32, Pm.primaryRays + 2 * (size_t)p,
                     Pm.primaryHits + 5 * (size_t)p, F))
            return false;
        beginRay<true>(Pm, st, s, F.org, aoDirection(F, Pm.seed, p, smp), 0.0f, Pm.aoLength);
        return true;
    }
    __device__ void finish(uint32_t i, const RayState& s) const {
        if (s.best.prim != kInvalid) atomicAdd(&counts[list[i / P->spp]], 1u);
    }
};

template <bool COUNT>
__global__ void aoTraceKernel(TraceParams P, const uint32_t* list, const uint32_t* listCount, uint32_t* counts) {
    extern __shared__ uint32_t sstack[];
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    Stack st{sstack + threadIdx.x, P.globalStack + gtid, P.sharedDepth, P.globalDepth, P.globalStride, 0};
    AoSource src{&P, list, listCount, counts};
    refillLoop<true, true, COUNT>(P, st, src);
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
static grtError prepareTrace(Context* c, grtScene scene, grtGeometry geom, grtFuncTable table,
                             const grtTraceOptions* opt, TraceParams& P, bool* isScene, int* blockSize) {
    if ((scene != nullptr) == (geom != nullptr)) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = findBvh(scene ? (const void*)scene : (const void*)geom);
    if (!o) return GRT_ERROR_INVALID_PARAMETER;
    if (scene && o->primType != kPrimScene) return GRT_ERROR_INVALID_PARAMETER;
    if (geom && o->primType == kPrimScene) return GRT_ERROR_INVALID_PARAMETER;
    if (!o->built) return GRT_ERROR_NOT_BUILT;
    *isScene = scene != nullptr;
    P.target.nodes = (const float4*)o->nodes;
    P.target.leaves = o->leaves;
    P.target.primType = o->primType;
    P.target.geomType = o->geomType;
    P.target.empty = o->primCount == 0;
    P.maxSteps = 1u << 26;  // far above any legitimate walk; stops a corrupted (cyclic) hierarchy
    const float compact = (opt && opt->compactThreshold > 0.f) ? fminf(opt->compactThreshold, 1.f) : 0.5f;
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

template <bool ANY, bool COUNT>
static void traceKernelFor(bool scene, void (**k)(TraceParams)) {
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
        traceKernelFor<ANY, true>(isScene, &kernel);
    else
        traceKernelFor<ANY, false>(isScene, &kernel);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = (size_t)bs * P.sharedDepth * sizeof(uint32_t);
    LaunchShape L = persistentShape(c, kernel, bs, smem);
    L.blocks = std::min<int>(L.blocks, (int)ceilDiv(n, bs));
    e = bindGlobalStack(c, opt, L.blocks * bs, P);
    if (e != GRT_SUCCESS) return e;
    P.counter = nextCounter(c);
    GRT_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));
    kernel<<<L.blocks, bs, smem, s>>>(P);
    if (!ANY) refineKernel<<<smCount(c) * 4, 256, 0, s>>>(P);
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
        traceKernelFor<false, true>(isScene, &kernel);
    else
        traceKernelFor<false, false>(isScene, &kernel);
    const size_t smem = (size_t)bs * P.sharedDepth * sizeof(uint32_t);
    LaunchShape L = persistentShape(c, kernel, bs, smem);
    L.blocks = std::min<int>(L.blocks, (int)ceilDiv(rayCount, bs));
    L.blocks = std::max(1, std::min<int>(L.blocks, (int)(capacity / perBlock)));  // the grid shrinks to fit
    P.counter = reinterpret_cast<unsigned long long*>(base);
    P.globalStack = reinterpret_cast<uint32_t*>(static_cast<char*>(base) + kNoAllocStackOffset);
    P.globalStride = (uint32_t)(L.blocks * bs);
    cudaStream_t s = (cudaStream_t)stream;
    GRT_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));  // the work counter starts at zero
    kernel<<<L.blocks, bs, smem, s>>>(P);
    refineKernel<<<smCount(c) * 4, 256, 0, s>>>(P);
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
    const size_t smem = (size_t)bs * sh * sizeof(uint32_t);
    int threads = 0;
    void (*kernels[])(TraceParams) = {traceKernel<false, false, false>, traceKernel<false, true, false>,
                                      traceKernel<true, false, false>,  traceKernel<true, true, false>,
                                      traceKernel<false, false, true>,  traceKernel<false, true, true>,
                                      traceKernel<true, false, true>,   traceKernel<true, true, true>};
    for (auto k : kernels) threads = std::max(threads, persistentShape(c, k, bs, smem).blocks * bs);
    threads = std::max(threads, persistentShape(c, aoTraceKernel<false>, bs, smem).blocks * bs);
    threads = std::max(threads, persistentShape(c, aoTraceKernel<true>, bs, smem).blocks * bs);
    *sizeBytes = (size_t)threads * gl * sizeof(uint32_t);
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
    grtError e = prepareTrace(c, scene, nullptr, nullptr, options, P, &isScene, &bs);
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
    void (*kernel)(TraceParams, const uint32_t*, const uint32_t*, uint32_t*) =
        count ? aoTraceKernel<true> : aoTraceKernel<false>;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = (size_t)bs * P.sharedDepth * sizeof(uint32_t);
    LaunchShape L = persistentShape(c, kernel, bs, smem);
    // scratch after the global stack: the hit count (256 B) and the list of hit pixels
    void* extra = nullptr;
    e = bindGlobalStack(c, options, L.blocks * bs, P, 256 + 4 * (size_t)pixelCount, &extra);
    if (e != GRT_SUCCESS) return e;
    uint32_t* listCount = static_cast<uint32_t*>(extra);
    uint32_t* list = reinterpret_cast<uint32_t*>(static_cast<char*>(extra) + 256);
    uint32_t* counts = reinterpret_cast<uint32_t*>(ao);
    P.counter = nextCounter(c);
    GRT_CUDA(cudaMemsetAsync(P.counter, 0, sizeof(unsigned long long), s));
    GRT_CUDA(cudaMemsetAsync(listCount, 0, sizeof(uint32_t), s));
    aoCompactKernel<<<ceilDiv(pixelCount, 256), 256, 0, s>>>((const uint32_t*)primaryHits, pixelCount, list, listCount,
                                                            counts);
    kernel<<<L.blocks, bs, smem, s>>>(P, list, listCount, counts);
    aoFinishKernel<<<smCount(c) * 4, 256, 0, s>>>(list, listCount, samplesPerPixel, ao);
    GRT_LAUNCH_CHECK();
    noteLaunches(3);
    return GRT_SUCCESS;
}

}  // extern "C"
