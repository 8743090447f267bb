// Context, object registry, function tables, error reporting and introspection.
// API shape: context creation and log level (paper Sec. 7.1), function table
// creation and assignment (Sec. 7.4); return-code checking as the paper's
// checkHiprt pattern.
#include <atomic>
#include <cstdarg>
#include <mutex>
#include <unordered_map>

#include "grt_internal.cuh"

namespace grt {

struct Context {
    int device;
    int sms;
    DeviceWorkspace* dWork;
    unsigned nextSlot;
    void* scratch;        // traversal global-stack spill area (grown on demand)
    size_t scratchBytes;
    void* aux;            // buffers passed between the launches of one call (grown on demand)
    size_t auxBytes;
    std::mutex lock;
};

unsigned long long* nextCounter(Context* c) {
    std::lock_guard<std::mutex> g(c->lock);
    const unsigned slot = c->nextSlot++ % kCounterSlots;
    return &c->dWork->counters[slot];
}

grtError contextAux(Context* c, size_t bytes, void** ptr) {
    std::lock_guard<std::mutex> g(c->lock);
    if (bytes > c->auxBytes) {
        // Growing needs an idle device: the old area may still be in use by queued work.
        GRT_CUDA(cudaDeviceSynchronize());
        cudaFree(c->aux);
        c->aux = nullptr;
        c->auxBytes = 0;
        GRT_CUDA(cudaMalloc(&c->aux, bytes));
        c->auxBytes = bytes;
    }
    *ptr = c->aux;
    return GRT_SUCCESS;
}

grtError contextScratch(Context* c, size_t bytes, void** ptr) {
    std::lock_guard<std::mutex> g(c->lock);
    if (bytes > c->scratchBytes) {
        // Growing needs an idle device: the old area may still be in use by queued work.
        GRT_CUDA(cudaDeviceSynchronize());
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratchBytes = 0;
        GRT_CUDA(cudaMalloc(&c->scratch, bytes));
        c->scratchBytes = bytes;
    }
    *ptr = c->scratch;
    return GRT_SUCCESS;
}

static int g_logLevel = GRT_LOG_ERROR | GRT_LOG_WARN;
static std::mutex g_mutex;
static std::unordered_map<const void*, BvhObject*> g_bvh;
static std::unordered_map<const void*, FuncTableObject*> g_tables;

static std::atomic<unsigned long long> g_launches{0};

int logLevel() { return g_logLevel; }
void noteLaunches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launchCountNow() { return g_launches.load(); }

void logf(int level, const char* fmt, ...) {
    if (!(g_logLevel & level)) return;
    va_list ap;
    va_start(ap, fmt);
    fprintf(stderr, "[grt %s] ", level == GRT_LOG_ERROR ? "error" : (level == GRT_LOG_WARN ? "warn" : "info"));
    vfprintf(stderr, fmt, ap);
    fputc('\n', stderr);
    va_end(ap);
}

Context* asContext(grtContext c) { return reinterpret_cast<Context*>(c); }
DeviceWorkspace* workspace(Context* c) { return c->dWork; }
int smCount(Context* c) { return c->sms; }
int deviceOf(Context* c) { return c->device; }

BvhObject* findBvh(const void* handle) {
    std::lock_guard<std::mutex> g(g_mutex);
    auto it = g_bvh.find(handle);
    return it == g_bvh.end() ? nullptr : it->second;
}
grtError registerBvh(BvhObject* obj) {
    std::lock_guard<std::mutex> g(g_mutex);
    g_bvh[obj->dHeader] = obj;
    return GRT_SUCCESS;
}
void unregisterBvh(const void* handle) {
    std::lock_guard<std::mutex> g(g_mutex);
    g_bvh.erase(handle);
}
FuncTableObject* findFuncTable(grtFuncTable t) {
    std::lock_guard<std::mutex> g(g_mutex);
    auto it = g_tables.find(t);
    return it == g_tables.end() ? nullptr : it->second;
}

uint32_t resolveMortonBits(uint32_t count, const grtBuildOptions* opt) {
    uint32_t b = opt ? opt->mortonBits : 0;
    if (b == 30 || b == 63) return b;
    return count <= (1u << 20) ? 30u : 63u;
}

BuildLayout buildLayout(uint32_t count, uint32_t mortonBits, bool scene) {
    BuildLayout L{};
    const size_t n = count ? count : 1;
    L.keyBytes = mortonBits == 30 ? 4 : 8;
    L.passes = (int)((mortonBits + 7) / 8);
    L.finalBuf = L.passes & 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = alignUp(off + bytes, 256);
        return o;
    };
    L.bounds = take(64);
    L.centroids = take(16 * n);
    L.keys[0] = take(L.keyBytes * n);
    L.keys[1] = take(L.keyBytes * n);
    L.vals[0] = take(4 * n);
    L.vals[1] = take(4 * n);
    L.hist = take(sortScratchBytes(count));
    L.flags = take(4 * n);
    L.extra = scene ? take(32 * n + sizeof(InstanceRecord) * n) : off;
    L.total = off;
    return L;
}

}  // namespace grt

using namespace grt;

extern "C" {

grtError grtCreateContext(uint32_t apiVersion, const grtContextCreationInput* input, grtContext* out) {
    if (apiVersion != GRT_API_VERSION) return GRT_ERROR_INVALID_API_VERSION;
    if (!input || !out) return GRT_ERROR_INVALID_PARAMETER;
    int ndev = 0;
    GRT_CUDA(cudaGetDeviceCount(&ndev));
    if (input->device < 0 || input->device >= ndev) return GRT_ERROR_INVALID_PARAMETER;
    GRT_CUDA(cudaSetDevice(input->device));
    Context* c = new Context();
    c->device = input->device;
    c->nextSlot = 0;
    c->scratch = nullptr;
    c->scratchBytes = 0;
    c->aux = nullptr;
    c->auxBytes = 0;
    cudaError_t e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, input->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->dWork, sizeof(DeviceWorkspace));
    if (e == cudaSuccess) e = cudaMemset(c->dWork, 0, sizeof(DeviceWorkspace));
    if (e != cudaSuccess) {
        logf(GRT_LOG_ERROR, "context creation: %s", cudaGetErrorString(e));
        delete c;
        return e == cudaErrorMemoryAllocation ? GRT_ERROR_OUT_OF_MEMORY : GRT_ERROR_CUDA;
    }
    *out = reinterpret_cast<grtContext>(c);
    return GRT_SUCCESS;
}

grtError grtDestroyContext(grtContext ctx) {
    if (!ctx) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    cudaFree(c->dWork);
    cudaFree(c->scratch);
    cudaFree(c->aux);
    delete c;
    return GRT_SUCCESS;
}

grtError grtSetLogLevel(uint32_t levels) {
    g_logLevel = (int)levels;
    return GRT_SUCCESS;
}

grtError grtGetLastDeviceError(grtContext ctx, void* stream, grtError* err) {
    if (!ctx || !err) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t v = 0;
    GRT_CUDA(cudaMemcpyAsync(&v, &c->dWork->error, sizeof(v), cudaMemcpyDeviceToHost, s));
    GRT_CUDA(cudaMemsetAsync(&c->dWork->error, 0, sizeof(uint32_t), s));
    GRT_CUDA(cudaStreamSynchronize(s));
    *err = (grtError)v;
    return GRT_SUCCESS;
}

grtError grtGetLaunchCount(uint64_t* count) {
    if (!count) return GRT_ERROR_INVALID_PARAMETER;
    *count = g_launches.load();
    return GRT_SUCCESS;
}

grtError grtGetTraceStatistics(grtContext ctx, void* stream, grtTraceStatistics* stats) {
    if (!ctx || !stats) return GRT_ERROR_INVALID_PARAMETER;
    Context* c = asContext(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
    GRT_CUDA(cudaMemcpyAsync(v, c->dWork->stats, sizeof(v), cudaMemcpyDeviceToHost, s));
    GRT_CUDA(cudaMemsetAsync(c->dWork->stats, 0, sizeof(v), s));
    GRT_CUDA(cudaStreamSynchronize(s));
    stats->rays = v[0];
    stats->nodesVisited = v[1];
    stats->trianglesTested = v[2];
    stats->customTested = v[3];
    stats->instancesEntered = v[4];
    stats->fp64Tests = v[5];
    return GRT_SUCCESS;
}

grtError grtCreateFuncTable(grtContext ctx, uint32_t numGeomTypes, uint32_t numRayTypes, grtFuncTable* out) {
    if (!ctx || !out || numGeomTypes == 0 || numRayTypes == 0 || numGeomTypes > 65536 || numRayTypes > 65536)
        return GRT_ERROR_INVALID_PARAMETER;
    FuncTableObject* t = new FuncTableObject();
    t->numGeomTypes = numGeomTypes;
    t->numRayTypes = numRayTypes;
    t->userEntry.assign((size_t)numGeomTypes * numRayTypes, 0);
    const size_t bytes = sizeof(FuncEntry) * numGeomTypes * numRayTypes;
    cudaError_t e = cudaMalloc(&t->dEntries, bytes);
    if (e == cudaSuccess) e = cudaMemset(t->dEntries, 0, bytes);
    if (e != cudaSuccess) {
        delete t;
        return GRT_ERROR_OUT_OF_MEMORY;
    }
    {
        std::lock_guard<std::mutex> g(g_mutex);
        g_tables[t->dEntries] = t;
    }
    *out = reinterpret_cast<grtFuncTable>(t->dEntries);
    return GRT_SUCCESS;
}

grtError grtSetFuncTable(grtContext ctx, grtFuncTable table, uint32_t geomType, uint32_t rayType, grtFuncDataSet set) {
    FuncTableObject* t = findFuncTable(table);
    if (!ctx || !t || geomType >= t->numGeomTypes || rayType >= t->numRayTypes) return GRT_ERROR_INVALID_PARAMETER;
    const bool userFunc = set.intersectFunc >= GRT_INTERSECT_USER, userFilter = set.filterFunc >= GRT_FILTER_USER;
    if ((set.intersectFunc > GRT_INTERSECT_SPHERE && !userFunc) ||
        (set.filterFunc > GRT_FILTER_PRIMITIVE_MASK && !userFilter))
        return GRT_ERROR_INVALID_PARAMETER;
    if (set.filterFunc == GRT_FILTER_PRIMITIVE_MASK && !set.filterFuncData) return GRT_ERROR_INVALID_PARAMETER;
    FuncEntry e{set.intersectFunc, set.filterFunc, set.intersectFuncData, set.filterFuncData};
    const size_t slot = (size_t)rayType * t->numGeomTypes + geomType;
    // Synchronous copy: the table may be used by work enqueued afterwards on any stream.
    GRT_CUDA(cudaMemcpy(t->dEntries + slot, &e, sizeof(e), cudaMemcpyHostToDevice));
    std::lock_guard<std::mutex> g(g_mutex);
    const uint8_t user = (userFunc || userFilter) ? 1 : 0;
    t->userEntries += user;
    t->userEntries -= t->userEntry[slot];
    t->userEntry[slot] = user;
    return GRT_SUCCESS;
}

grtError grtDestroyFuncTable(grtContext ctx, grtFuncTable table) {
    FuncTableObject* t = findFuncTable(table);
    if (!ctx || !t) return GRT_ERROR_INVALID_PARAMETER;
    {
        std::lock_guard<std::mutex> g(g_mutex);
        g_tables.erase(table);
    }
    cudaFree(t->dEntries);
    delete t;
    return GRT_SUCCESS;
}

grtError grtGetBvhInfo(grtContext ctx, grtGeometry geom, grtScene scene, grtBvhInfo* info) {
    if (!ctx || !info || ((geom != nullptr) == (scene != nullptr))) return GRT_ERROR_INVALID_PARAMETER;
    BvhObject* o = findBvh(geom ? (const void*)geom : (const void*)scene);
    if (!o) return GRT_ERROR_INVALID_PARAMETER;
    info->nodes = o->nodes;
    info->wideNodes = o->wide;
    info->quantNodes = o->quant ? o->qnodes : nullptr;
    info->wide8Nodes = o->wide8 ? o->w8nodes : nullptr;
    info->leaves = o->leaves;
    info->parents = o->parents;
    info->nodeCount = o->nodeCount;
    info->primCount = o->primCount;
    info->leafCount = o->leafCount;
    info->reserved = 0;
    info->primType = o->primType;
    info->mortonBits = o->mortonBits;
    return o->built ? GRT_SUCCESS : GRT_ERROR_NOT_BUILT;
}

grtError grtGetBuildTemporaryLayout(uint32_t count, uint32_t mortonBits, size_t* sortedKeysOffset,
                                    size_t* sortedValuesOffset, size_t* centroidBoundsOffset) {
    if (!sortedKeysOffset || !sortedValuesOffset || !centroidBoundsOffset) return GRT_ERROR_INVALID_PARAMETER;
    grtBuildOptions o{0, mortonBits, 0.f};
    const BuildLayout L = buildLayout(count, resolveMortonBits(count, &o), false);
    *sortedKeysOffset = L.keys[L.finalBuf];
    *sortedValuesOffset = L.vals[L.finalBuf];
    *centroidBoundsOffset = L.bounds;
    return GRT_SUCCESS;
}

}  // extern "C"
