// Serving runtime: a table of resident hierarchies and graph-replayed steps.
//
// Each step evaluates a list of segments (slices of requests, possibly on
// different maps) in one persistent kernel launch.  The segment table is
// written into a pinned host buffer and copied to the device by the step's
// CUDA graph (copy, cursor reset, kernel), captured once per table slot.
// Slots rotate: writing a slot's host buffer only waits for the step that last
// used that slot, so several steps can be queued while earlier ones run.
#include <math.h>
#include <string.h>

#include <new>

#include "area_step.cuh"
#include "common.cuh"

using namespace pndf;

namespace {

struct Slot {
    void *host = nullptr;            // pinned: header + prefix + segments
    void *dev = nullptr;             // device: same layout, then the work cursor
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool used = false;
};

size_t prefix_bytes(int max_segs) { return ((size_t(max_segs) + 2) * sizeof(uint32_t) + 15) & ~size_t(15); }

size_t pndf_table_bytes(int max_segs) { return prefix_bytes(max_segs) + size_t(max_segs) * sizeof(pndf_segment); }

// Step table: the P-NDF part (count, prefix sums, segments), then the
// projected-area part (count padded to 16 bytes, then one descriptor per
// request); both are copied to the device by the step graph.
size_t area_table_bytes(int area_cap) { return area_cap > 0 ? 16 + size_t(area_cap) * sizeof(AreaReq) : 0; }

size_t table_bytes(int max_segs, int area_cap) { return pndf_table_bytes(max_segs) + area_table_bytes(area_cap); }

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

struct pndf_server {
    int device = 0;
    int nmaps = 0;
    int texel_fmt = 0, bounds_fmt = 0;
    int max_segs = 0, warps = 8, ctas = 0;
    int kernel = PNDF_KERNEL_GAUSS;
    float tau = 0.f, jac_eps = 0.f;
    uint32_t split_cap = 0;  // entries of a step's division of large footprints (0: cluster cut, none)
    MapDesc *maps_dev = nullptr;
    ClusterDesc *clusters_dev = nullptr;  // per map, read only with tau > 0
    cudaStream_t cap = nullptr;
    int area_cap = 0;     // projected-area requests per step
    int area_bands = 0;   // bands per request at most (largest map)
    static constexpr int kMaxSlots = 8;
    Slot slot[kMaxSlots];
    int nslots = 4;
    int next = 0;
};

namespace {

void release(pndf_server *s)
{
    if (!s) return;
    for (Slot &sl : s->slot) {
        if (sl.done) cudaEventSynchronize(sl.done);
        if (!sl.host && !sl.dev && !sl.exec && !sl.done) continue;
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.host) cudaFreeHost(sl.host);
    }
    if (s->maps_dev) cudaFree(s->maps_dev);
    if (s->clusters_dev) cudaFree(s->clusters_dev);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

// Device bytes of a slot: the table, the P-NDF work cursor, the division of
// large footprints, and for the projected-area part the band offsets, band
// partial sums and their cursor.
size_t slot_device_bytes(const pndf_server *s)
{
    size_t b = up256(table_bytes(s->max_segs, s->area_cap)) + 256 + up256(serve_split_bytes(s->split_cap));
    if (s->area_cap > 0)
        b += up256((size_t(s->area_cap) + 1) * sizeof(uint32_t)) +
             up256(size_t(s->area_cap) * s->area_bands * sizeof(float2)) + 256;
    return b;
}

cudaError_t capture_slot(pndf_server *s, Slot &sl)
{
    const size_t tb = table_bytes(s->max_segs, s->area_cap);
    char *dev = static_cast<char *>(sl.dev);
    const uint32_t *table = reinterpret_cast<const uint32_t *>(dev);
    const pndf_segment *segs = reinterpret_cast<const pndf_segment *>(dev + prefix_bytes(s->max_segs));
    auto *cursor = reinterpret_cast<unsigned long long *>(dev + up256(tb));
    cudaError_t e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaMemcpyAsync(sl.dev, sl.host, tb, cudaMemcpyHostToDevice, s->cap);
    cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s->cap);
    const ServeVariant v{s->kernel, s->tau, s->jac_eps};
    char *split = dev + up256(tb) + 256;
    launch_serve(s->texel_fmt, s->bounds_fmt, v, s->maps_dev, s->clusters_dev, s->nmaps, table, segs, cursor,
                 s->warps, s->ctas, s->split_cap > 0 ? split : nullptr, s->split_cap, s->cap);
    if (s->area_cap > 0) {
        char *at = dev + pndf_table_bytes(s->max_segs);
        char *scratch = split + up256(serve_split_bytes(s->split_cap));
        auto *off = reinterpret_cast<uint32_t *>(scratch);
        scratch += up256((size_t(s->area_cap) + 1) * sizeof(uint32_t));
        auto *part = reinterpret_cast<float2 *>(scratch);
        scratch += up256(size_t(s->area_cap) * s->area_bands * sizeof(float2));
        launch_area_step(s->texel_fmt, s->maps_dev, s->nmaps, reinterpret_cast<const uint32_t *>(at),
                         reinterpret_cast<const AreaReq *>(at + 16), s->area_cap, off, part,
                         reinterpret_cast<unsigned int *>(scratch), s->cap);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ec = cudaStreamEndCapture(s->cap, &g);
    if (ec != cudaSuccess) return ec;
    e = cudaGraphInstantiate(&sl.exec, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

extern "C" {

pndf_status pndf_server_create(const pndf_hierarchy *const *maps, int32_t nmaps, const pndf_server_config *cfg,
                               pndf_server **out)
{
    if (!out) return PNDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!maps || nmaps < 1 || nmaps > kServeMaxMaps) return PNDF_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNDF_ERR_CUDA;
    for (int i = 0; i < nmaps; ++i) {
        if (!maps[i] || !maps[i]->mem || maps[i]->device != dev) return PNDF_ERR_INVALID_ARG;
        if (maps[i]->d.texel_fmt != maps[0]->d.texel_fmt || maps[i]->d.bounds_fmt != maps[0]->d.bounds_fmt)
            return PNDF_ERR_INVALID_ARG;
    }
    pndf_server_config c{1024, 8, 0, 4, PNDF_KERNEL_GAUSS, 0.f, 0.f, 0};
    if (cfg) {
        if (cfg->max_segments < 0 || cfg->warps_per_cta < 0 || cfg->warps_per_cta > 8 || cfg->ctas_per_sm < 0 ||
            cfg->slots < 0 || cfg->slots == 1 || cfg->slots > pndf_server::kMaxSlots ||
            cfg->max_area_requests < 0 || cfg->max_area_requests > 65536)
            return PNDF_ERR_INVALID_ARG;
        c.max_area_requests = cfg->max_area_requests;
        if (cfg->kernel != PNDF_KERNEL_GAUSS && cfg->kernel != PNDF_KERNEL_DISK && cfg->kernel != PNDF_KERNEL_BOX)
            return PNDF_ERR_INVALID_ARG;
        if (!(cfg->tau >= 0.f) || !isfinite(cfg->tau)) return PNDF_ERR_INVALID_ARG;
        if (!(cfg->jac_eps == 0.f || (cfg->jac_eps >= 1e-9f && cfg->jac_eps <= 1e-2f))) return PNDF_ERR_INVALID_ARG;
        if (cfg->max_segments) c.max_segments = cfg->max_segments;
        if (cfg->warps_per_cta) c.warps_per_cta = cfg->warps_per_cta;
        if (cfg->slots) c.slots = cfg->slots;
        c.ctas_per_sm = cfg->ctas_per_sm;
        c.kernel = cfg->kernel;
        c.tau = cfg->tau;
        c.jac_eps = cfg->jac_eps;
    }
    if (c.max_segments > (1 << 16)) return PNDF_ERR_INVALID_ARG;
    if (c.tau > 0.f) {
        if (c.kernel != PNDF_KERNEL_GAUSS || c.jac_eps > 0.f) return PNDF_ERR_UNSUPPORTED;
        for (int i = 0; i < nmaps; ++i)
            if (!maps[i]->clusters) return PNDF_ERR_UNSUPPORTED;
    }
    if (c.jac_eps > 0.f && c.kernel != PNDF_KERNEL_GAUSS) return PNDF_ERR_UNSUPPORTED;
    pndf_server *s = new (std::nothrow) pndf_server();
    if (!s) return PNDF_ERR_OOM;
    s->device = dev;
    s->nmaps = nmaps;
    s->texel_fmt = maps[0]->d.texel_fmt;
    s->bounds_fmt = maps[0]->d.bounds_fmt;
    s->max_segs = c.max_segments;
    s->warps = c.warps_per_cta;
    s->ctas = c.ctas_per_sm;
    s->nslots = c.slots;
    s->kernel = c.kernel;
    s->tau = c.tau;
    s->jac_eps = c.jac_eps;
    s->area_cap = c.max_area_requests;
    s->split_cap = c.tau > 0.f ? 0u : serve_split_cap();
    for (int i = 0; i < nmaps; ++i) s->area_bands = max(s->area_bands, area_max_bands(maps[i]->d.n));
    MapDesc host_maps[kServeMaxMaps];
    ClusterDesc host_clusters[kServeMaxMaps];
    for (int i = 0; i < nmaps; ++i) {
        host_maps[i] = maps[i]->d;
        host_clusters[i] = maps[i]->c;
    }
    const size_t tb = table_bytes(s->max_segs, s->area_cap);
    bool ok = cudaMalloc(&s->maps_dev, sizeof(MapDesc) * nmaps) == cudaSuccess &&
              cudaMemcpy(s->maps_dev, host_maps, sizeof(MapDesc) * nmaps, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMalloc(&s->clusters_dev, sizeof(ClusterDesc) * nmaps) == cudaSuccess &&
              cudaMemcpy(s->clusters_dev, host_clusters, sizeof(ClusterDesc) * nmaps, cudaMemcpyHostToDevice) ==
                  cudaSuccess &&
              cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) == cudaSuccess &&
              prepare_serve(s->texel_fmt, s->bounds_fmt, ServeVariant{s->kernel, s->tau, s->jac_eps}, s->warps) ==
                  cudaSuccess;
    for (int k = 0; ok && k < s->nslots; ++k) {
        Slot &sl = s->slot[k];
        ok = cudaMallocHost(&sl.host, tb) == cudaSuccess && cudaMalloc(&sl.dev, slot_device_bytes(s)) == cudaSuccess &&
             cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
        if (ok) {
            memset(sl.host, 0, tb);
            ok = capture_slot(s, sl) == cudaSuccess;
        }
    }
    if (!ok) {
        cudaError_t e = cudaGetLastError();
        release(s);
        return e == cudaErrorMemoryAllocation ? PNDF_ERR_OOM : PNDF_ERR_CUDA;
    }
    *out = s;
    return PNDF_OK;
}

pndf_status pndf_server_step(pndf_server *s, const pndf_segment *segs, int32_t nsegs, void *stream, void *ev_done)
{
    if (!s) return PNDF_ERR_INVALID_ARG;
    if (nsegs < 0 || (nsegs > 0 && !segs)) return PNDF_ERR_INVALID_ARG;
    uint64_t total = 0;
    int npndf = 0;
    int64_t narea = 0;
    for (int i = 0; i < nsegs; ++i) {
        const pndf_segment &g = segs[i];
        if (g.map < 0 || g.map >= s->nmaps || g.count < 0 || g.first < 0) return PNDF_ERR_INVALID_ARG;
        if (g.count > 0 && (!g.q || !g.D)) return PNDF_ERR_INVALID_ARG;
        if (g.kind == PNDF_SEGMENT_PNDF) {
            total += uint64_t(g.count);
            ++npndf;
        } else if (g.kind == PNDF_SEGMENT_PROJECTED_AREA) {
            if (g.order || g.flags || (g.count > 0 && (!g.omega || (reinterpret_cast<uintptr_t>(g.omega) & 3u))))
                return PNDF_ERR_INVALID_ARG;
            narea += g.count;
        } else {
            return PNDF_ERR_INVALID_ARG;
        }
    }
    if (npndf > s->max_segs || total >= (uint64_t(1) << 32)) return PNDF_ERR_INVALID_ARG;
    if (narea > s->area_cap) return narea > 0 && s->area_cap == 0 ? PNDF_ERR_UNSUPPORTED : PNDF_ERR_CAPACITY;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device) return PNDF_ERR_INVALID_ARG;
    Slot &sl = s->slot[s->next];
    s->next = (s->next + 1) % s->nslots;
    if (sl.used && cudaEventSynchronize(sl.done) != cudaSuccess) return PNDF_ERR_CUDA;
    uint32_t *hdr = static_cast<uint32_t *>(sl.host);
    hdr[0] = uint32_t(npndf);
    uint32_t *prefix = hdr + 1;
    prefix[0] = 0;
    auto *ptab = reinterpret_cast<pndf_segment *>(static_cast<char *>(sl.host) + prefix_bytes(s->max_segs));
    int k = 0;
    for (int i = 0; i < nsegs; ++i)
        if (segs[i].kind == PNDF_SEGMENT_PNDF) {
            ptab[k] = segs[i];
            prefix[k + 1] = prefix[k] + uint32_t(segs[i].count);
            ++k;
        }
    if (s->area_cap > 0) {
        char *at = static_cast<char *>(sl.host) + pndf_table_bytes(s->max_segs);
        auto *areq = reinterpret_cast<AreaReq *>(at + 16);
        uint32_t na = 0;
        for (int i = 0; i < nsegs; ++i) {
            const pndf_segment &g = segs[i];
            if (g.kind != PNDF_SEGMENT_PROJECTED_AREA) continue;
            for (int32_t r = 0; r < g.count; ++r, ++na)
                areq[na] = AreaReq{g.q + g.first + r, g.omega + 3 * (size_t(g.first) + r), g.D + g.first + r, g.map, 0};
        }
        *reinterpret_cast<uint32_t *>(at) = na;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGraphLaunch(sl.exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
    if (e == cudaSuccess && ev_done) e = cudaEventRecord(static_cast<cudaEvent_t>(ev_done), st);
    sl.used = true;
    count_launches(1);
    return e == cudaSuccess ? PNDF_OK : PNDF_ERR_CUDA;
}

pndf_status pndf_server_sync(pndf_server *s)
{
    if (!s) return PNDF_ERR_INVALID_ARG;
    for (Slot &sl : s->slot)
        if (sl.used && cudaEventSynchronize(sl.done) != cudaSuccess) return PNDF_ERR_CUDA;
    return PNDF_OK;
}

void pndf_server_destroy(pndf_server *s)
{
    if (!s) return;
    int cur = -1;
    cudaGetDevice(&cur);
    const int dev = s->device;
    if (cur != dev) cudaSetDevice(dev);  // its memory, streams and graphs belong to its device
    release(s);
    if (cur != dev && cur >= 0) cudaSetDevice(cur);
}

}  // extern "C"
