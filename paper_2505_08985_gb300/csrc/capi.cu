// C ABI entry points of libpndf.so (declarations and contracts in pndf.h).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>

#include "common.cuh"
#include "ggx.cuh"
#include "shard.cuh"

using namespace pndf;

namespace {

std::atomic<int64_t> g_launches{0};


cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Keep stream-ordered scratch cached in the device's default pool instead of
// releasing it to the operating system at every synchronisation (once per device).
void keep_pool_memory()
{
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return;
    uint64_t bit = uint64_t(1) << dev;
    if (done.fetch_or(bit) & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
}

// The address at which the current device reads a texel array: device
// memory of this device as is, page-locked host memory through its mapped
// device address (the build kernel then reads the map straight over the host
// link, with no staging copy); nullptr for anything else (pageable host
// memory, another device's memory), which the entry points reject before any
// work is queued.
const void *device_view(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device == dev ? p : nullptr;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

pndf_status check_hierarchy(const pndf_hierarchy *h)
{
    if (!h || !h->mem) return PNDF_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PNDF_ERR_CUDA;
    if (dev != h->device) return PNDF_ERR_INVALID_ARG;  // must be called with the hierarchy's device current
    keep_pool_memory();
    return PNDF_OK;
}

// Status read-out: kernels that take a status word (atomic exchange with 0)
// write the old value into this page-locked, mapped host buffer; a mutex
// orders the callers, which wait on their stream before reading.
std::mutex g_status_mutex;
unsigned int *g_status_host = nullptr;  // 4 words

__global__ void take_word(unsigned int *word, unsigned int *out) { *out = atomicExch(word, 0u); }

cudaError_t status_buffer(unsigned int **host, unsigned int **dev)
{
    if (!g_status_host) {
        void *p = nullptr;
        cudaError_t e = cudaHostAlloc(&p, 4 * sizeof(unsigned int), cudaHostAllocPortable | cudaHostAllocMapped);
        if (e != cudaSuccess) return e;
        g_status_host = static_cast<unsigned int *>(p);
    }
    *host = g_status_host;
    return cudaHostGetDevicePointer(reinterpret_cast<void **>(dev), g_status_host, 0);
}

}  // namespace

void pndf::count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" {

pndf_status pndf_build_hierarchy(const void *texels_dev, const pndf_build_params *p, void *stream,
                                 pndf_hierarchy **out)
{
    if (!out) return PNDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!texels_dev || !p) return PNDF_ERR_INVALID_ARG;
    if (p->n < 2 || p->n > 16384) return PNDF_ERR_INVALID_ARG;
    if (p->texel_fmt != PNDF_TEXEL_F32X2 && p->texel_fmt != PNDF_TEXEL_F16X2) return PNDF_ERR_INVALID_ARG;
    if (p->bounds_fmt != PNDF_BOUNDS_F32 && p->bounds_fmt != PNDF_BOUNDS_F16_OUTWARD) return PNDF_ERR_INVALID_ARG;
    if (p->leaf_level != 0 && p->leaf_level != kLeafLevel) return PNDF_ERR_UNSUPPORTED;
    if (p->clusters != 0 && p->clusters != 1) return PNDF_ERR_INVALID_ARG;
    if (!aligned(texels_dev, p->texel_fmt == PNDF_TEXEL_F32X2 ? 8 : 4)) return PNDF_ERR_INVALID_ARG;
    const void *src = device_view(texels_dev);
    if (!src) return PNDF_ERR_INVALID_ARG;

    pndf_hierarchy *h = new (std::nothrow) pndf_hierarchy();
    if (!h) return PNDF_ERR_OOM;
    memset(&h->d, 0, sizeof(h->d));
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return PNDF_ERR_CUDA;
    }
    MapDesc &d = h->d;
    d.n = p->n;
    d.L = top_level(p->n);
    d.texel_fmt = p->texel_fmt;
    d.bounds_fmt = p->bounds_fmt;
    const size_t node_b = p->bounds_fmt == PNDF_BOUNDS_F32 ? 16 : 8;
    const size_t texel_b = p->texel_fmt == PNDF_TEXEL_F32X2 ? 8 : 4;
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    size_t off[kMaxLevels + 1];
    size_t total = up(size_t(d.n) * d.n * texel_b);
    off[0] = total;  // level 0: one box per quad
    total += up(level_nodes(d.L, 0) * node_b);
    const size_t off_qcap = total;  // and one capsule per quad
    total += up(level_nodes(d.L, 0) * sizeof(uint2));
    for (int l = kLeafLevel; l <= d.L; ++l) {
        off[l] = total;
        total += up(level_nodes(d.L, l) * node_b);
    }
    // cluster records (two float4 per node), residuals, build scratch
    size_t off_cl[kMaxLevels], off_ce[kMaxLevels], off_mom = 0;
    h->clusters = p->clusters;
    if (h->clusters) {
        for (int l = kLeafLevel; l <= d.L; ++l) {
            off_cl[l] = total;
            total += up(level_nodes(d.L, l) * 2 * sizeof(float4));
            off_ce[l] = total;
            total += up(level_nodes(d.L, l) * sizeof(float));
        }
        off_mom = total;
        total += up(cluster_scratch_bytes(d.L));
    }
    const size_t off_status = total;  // the hierarchy's status word
    total += 256;
    if (cudaMalloc(&h->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return PNDF_ERR_OOM;
    }
    h->bytes = total;
    char *base = static_cast<char *>(h->mem);
    d.texels = base;
    d.lv[0] = base + off[0];
    d.qcap = reinterpret_cast<const uint2 *>(base + off_qcap);
    for (int l = kLeafLevel; l <= d.L; ++l) d.lv[l] = base + off[l];
    memset(&h->c, 0, sizeof(h->c));
    h->moments = nullptr;
    if (h->clusters) {
        for (int l = kLeafLevel; l <= d.L; ++l) {
            h->c.cl[l] = reinterpret_cast<const float4 *>(base + off_cl[l]);
            h->c.ce[l] = reinterpret_cast<const float *>(base + off_ce[l]);
        }
        if (cluster_scratch_bytes(d.L)) h->moments = base + off_mom;
    }
    d.status = reinterpret_cast<unsigned int *>(base + off_status);
    cudaError_t e = cudaMemsetAsync(d.status, 0, sizeof(unsigned int), as_stream(stream));
    if (e == cudaSuccess) e = launch_build(src, h, as_stream(stream));
    if (e != cudaSuccess) {
        cudaFree(h->mem);
        delete h;
        return PNDF_ERR_CUDA;
    }
    *out = h;
    return PNDF_OK;
}

pndf_status pndf_update_hierarchy(pndf_hierarchy *h, const void *texels_dev, void *stream)
{
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    if (!texels_dev || !aligned(texels_dev, h->d.texel_fmt == PNDF_TEXEL_F32X2 ? 8 : 4)) return PNDF_ERR_INVALID_ARG;
    const void *src = device_view(texels_dev);
    if (!src) return PNDF_ERR_INVALID_ARG;
    return launch_build(src, h, as_stream(stream)) == cudaSuccess ? PNDF_OK : PNDF_ERR_CUDA;
}

void pndf_free_hierarchy(pndf_hierarchy *h)
{
    if (!h) return;
    if (h->mem) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != h->device) cudaSetDevice(h->device);
        cudaFree(h->mem);
        if (cur != h->device && cur >= 0) cudaSetDevice(cur);
    }
    delete h;
}

size_t pndf_hierarchy_bytes(const pndf_hierarchy *h) { return h ? h->bytes : 0; }

pndf_status pndf_sample_normals(const pndf_hierarchy *h, const pndf_query *q_dev, const float *u_dev, int64_t n,
                                int32_t kernel, float jac_eps, float *m_out_dev, uint32_t *tri_out_dev,
                                uint32_t *flags_out_dev, void *stream)
{
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    if (n < 0 || (n > 0 && (!q_dev || !u_dev || !m_out_dev))) return PNDF_ERR_INVALID_ARG;
    if ((q_dev && !aligned(q_dev, 16)) || (u_dev && !aligned(u_dev, 4)) || (m_out_dev && !aligned(m_out_dev, 4)))
        return PNDF_ERR_INVALID_ARG;
    if (kernel != PNDF_KERNEL_GAUSS && kernel != PNDF_KERNEL_DISK && kernel != PNDF_KERNEL_BOX)
        return PNDF_ERR_INVALID_ARG;
    if (!(jac_eps == 0.f || (jac_eps >= 1e-9f && jac_eps <= 1e-2f))) return PNDF_ERR_INVALID_ARG;
    return launch_sample(h, q_dev, u_dev, n, kernel, jac_eps, m_out_dev, tri_out_dev, flags_out_dev,
                         as_stream(stream)) == cudaSuccess
               ? PNDF_OK
               : PNDF_ERR_CUDA;
}

pndf_status pndf_ggx_create(const pndf_hierarchy *h, void *stream, pndf_ggx **out)
{
    if (!out) return PNDF_ERR_INVALID_ARG;
    *out = nullptr;
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    pndf_ggx *g = new (std::nothrow) pndf_ggx();
    if (!g) return PNDF_ERR_OOM;
    memset(g, 0, sizeof(*g));
    g->device = h->device;
    g->n = h->d.n;
    g->L = h->d.L;
    size_t off[kMaxLevels] = {0}, total = 0;
    for (int l = kLeafLevel; l <= g->L; ++l) {
        off[l] = total;
        total += (level_nodes(g->L, l) * sizeof(float4) + 255) & ~size_t(255);
    }
    if (cudaMalloc(&g->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return PNDF_ERR_OOM;
    }
    g->bytes = total;
    for (int l = kLeafLevel; l <= g->L; ++l) g->omega[l] = reinterpret_cast<float4 *>(static_cast<char *>(g->mem) + off[l]);
    st = launch_ggx_build(h, g, as_stream(stream));
    if (st != PNDF_OK) {
        cudaFree(g->mem);
        delete g;
        return st;
    }
    *out = g;
    return PNDF_OK;
}

void pndf_ggx_free(pndf_ggx *g)
{
    if (!g) return;
    if (g->mem) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != g->device) cudaSetDevice(g->device);
        cudaFree(g->mem);
        if (cur != g->device && cur >= 0) cudaSetDevice(cur);
    }
    delete g;
}

static pndf_status ggx_args(const pndf_ggx *g, const pndf_query *q, const float *a, const float *b, int64_t n,
                            const float *out, bool need_b)
{
    if (!g || !g->mem || n < 0) return PNDF_ERR_INVALID_ARG;
    if (n > 0 && (!q || !a || !out || (need_b && !b))) return PNDF_ERR_INVALID_ARG;
    if ((q && !aligned(q, 16)) || (a && !aligned(a, 4)) || (b && !aligned(b, 4)) || (out && !aligned(out, 4)))
        return PNDF_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device) return PNDF_ERR_INVALID_ARG;
    return PNDF_OK;
}

pndf_status pndf_ggx_lambda(const pndf_ggx *g, const pndf_query *q_dev, const float *omega_dev, int64_t n,
                            float *lambda_out_dev, void *stream)
{
    pndf_status st = ggx_args(g, q_dev, omega_dev, nullptr, n, lambda_out_dev, false);
    if (st != PNDF_OK) return st;
    return launch_ggx_eval(g, q_dev, omega_dev, nullptr, n, lambda_out_dev, as_stream(stream)) == cudaSuccess
               ? PNDF_OK
               : PNDF_ERR_CUDA;
}

pndf_status pndf_shadow_masking(const pndf_ggx *g, const pndf_query *q_dev, const float *wi_dev,
                                const float *wo_dev, int64_t n, float *G_out_dev, void *stream)
{
    pndf_status st = ggx_args(g, q_dev, wi_dev, wo_dev, n, G_out_dev, true);
    if (st != PNDF_OK) return st;
    return launch_ggx_eval(g, q_dev, wi_dev, wo_dev, n, G_out_dev, as_stream(stream)) == cudaSuccess ? PNDF_OK
                                                                                                     : PNDF_ERR_CUDA;
}

pndf_status pndf_ggx_level(const pndf_ggx *g, int32_t level, float *omega_out_dev, void *stream)
{
    if (!g || !g->mem || level < kLeafLevel || level > g->L || !omega_out_dev || !aligned(omega_out_dev, 4))
        return PNDF_ERR_INVALID_ARG;
    return launch_ggx_copy(g, level, omega_out_dev, as_stream(stream)) == cudaSuccess ? PNDF_OK : PNDF_ERR_CUDA;
}

pndf_status pndf_cluster_level(const pndf_hierarchy *h, int32_t level, float *records_dev, float *residual_dev,
                               void *stream)
{
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    if (!h->clusters) return PNDF_ERR_UNSUPPORTED;
    if (level < kLeafLevel || level > h->d.L || !records_dev || !residual_dev) return PNDF_ERR_INVALID_ARG;
    if (!aligned(records_dev, 4) || !aligned(residual_dev, 4)) return PNDF_ERR_INVALID_ARG;
    return launch_cluster_copy(h, level, records_dev, residual_dev, as_stream(stream)) == cudaSuccess ? PNDF_OK
                                                                                                    : PNDF_ERR_CUDA;
}

pndf_status pndf_eval_batch_ex(const pndf_hierarchy *h, const pndf_query *q_dev, int64_t nq, float *D_out_dev,
                               uint32_t *flags_out_dev, pndf_query_stats *stats_dev, const pndf_eval_config *cfg,
                               void *stream)
{
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    if (nq < 0 || nq > int64_t(0x7fffffff)) return PNDF_ERR_INVALID_ARG;
    if (nq > 0 && (!q_dev || !D_out_dev)) return PNDF_ERR_INVALID_ARG;
    if (q_dev && !aligned(q_dev, 16)) return PNDF_ERR_INVALID_ARG;
    pndf_eval_config c{PNDF_MODE_HIERARCHY, PNDF_SORT_DEFAULT, 0, 0, 0.f, PNDF_KERNEL_GAUSS, 0.f, 0, nullptr, nullptr};
    if (cfg) c = *cfg;
    if (c.mode != PNDF_MODE_HIERARCHY && c.mode != PNDF_MODE_FLAT) return PNDF_ERR_INVALID_ARG;
    if (!(c.tau >= 0.f) || !isfinite(c.tau)) return PNDF_ERR_INVALID_ARG;
    if (c.kernel != PNDF_KERNEL_GAUSS && c.kernel != PNDF_KERNEL_DISK && c.kernel != PNDF_KERNEL_BOX)
        return PNDF_ERR_INVALID_ARG;
    if (!(c.jac_eps == 0.f || (c.jac_eps >= 1e-9f && c.jac_eps <= 1e-2f)) || !(c.split == 0 || c.split == -1))
        return PNDF_ERR_INVALID_ARG;
    if (c.jac_eps > 0.f && (c.kernel != PNDF_KERNEL_GAUSS || c.mode != PNDF_MODE_HIERARCHY || c.tau > 0.f))
        return PNDF_ERR_UNSUPPORTED;
    if (c.tau > 0.f && (!h->clusters || c.mode != PNDF_MODE_HIERARCHY)) return PNDF_ERR_UNSUPPORTED;
    if (c.sort < 0 || c.sort > 4) return PNDF_ERR_INVALID_ARG;
    if (c.warps_per_cta < 0 || c.warps_per_cta > 8 || c.ctas_per_sm < 0) return PNDF_ERR_INVALID_ARG;
    return launch_eval(h, q_dev, nq, D_out_dev, flags_out_dev, stats_dev, c, as_stream(stream));
}

pndf_status pndf_eval_batch(const pndf_hierarchy *h, const pndf_query *q_dev, int64_t nq, float *D_out_dev,
                            uint32_t *flags_out_dev, pndf_query_stats *stats_dev, void *stream)
{
    return pndf_eval_batch_ex(h, q_dev, nq, D_out_dev, flags_out_dev, stats_dev, nullptr, stream);
}

pndf_status pndf_eval_batch_noalloc(const pndf_hierarchy *h, const pndf_query *q_dev, int64_t nq, float *D_out_dev,
                                    uint32_t *flags_out_dev, void *stream)
{
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    if (nq < 0) return PNDF_ERR_INVALID_ARG;
    if (nq > noalloc_max_queries()) return PNDF_ERR_CAPACITY;
    if (nq > 0 && (!q_dev || !D_out_dev)) return PNDF_ERR_INVALID_ARG;
    if (q_dev && !aligned(q_dev, 16)) return PNDF_ERR_INVALID_ARG;
    return launch_eval_noalloc(h, q_dev, nq, D_out_dev, flags_out_dev, as_stream(stream));
}

int64_t pndf_eval_noalloc_max_queries(void) { return noalloc_max_queries(); }

pndf_status pndf_sort_queries(const pndf_hierarchy *h, const pndf_query *q_dev, int64_t nq, uint32_t *order_dev,
                              void *stream)
{
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    if (nq < 0 || nq > int64_t(0x7fffffff)) return PNDF_ERR_INVALID_ARG;
    if (nq > 0 && (!q_dev || !order_dev)) return PNDF_ERR_INVALID_ARG;
    if (q_dev && !aligned(q_dev, 16)) return PNDF_ERR_INVALID_ARG;
    return launch_sort(h, q_dev, nq, order_dev, as_stream(stream));
}

pndf_status pndf_eval_batch_host(const pndf_hierarchy *h, const pndf_query *q_host, int64_t nq, float *D_host,
                                 void *stream)
{
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    if (nq < 0 || nq > int64_t(0x7fffffff)) return PNDF_ERR_INVALID_ARG;
    if (nq == 0) return PNDF_OK;
    if (!q_host || !D_host) return PNDF_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    size_t qb = size_t(nq) * sizeof(pndf_query), db = size_t(nq) * sizeof(float);
    size_t qoff = (db + 255) & ~size_t(255);
    void *buf = nullptr;
    if (cudaMallocAsync(&buf, qoff + qb, s) != cudaSuccess) {
        cudaGetLastError();
        return PNDF_ERR_OOM;
    }
    float *Dd = static_cast<float *>(buf);
    pndf_query *qd = reinterpret_cast<pndf_query *>(static_cast<char *>(buf) + qoff);
    cudaError_t e = cudaMemcpyAsync(qd, q_host, qb, cudaMemcpyHostToDevice, s);
    pndf_eval_config c{PNDF_MODE_HIERARCHY, PNDF_SORT_DEFAULT, 0, 0, 0.f, PNDF_KERNEL_GAUSS, 0.f, 0, nullptr, nullptr};
    if (e == cudaSuccess) st = launch_eval(h, qd, nq, Dd, nullptr, nullptr, c, s);
    if (e == cudaSuccess && st == PNDF_OK) e = cudaMemcpyAsync(D_host, Dd, db, cudaMemcpyDeviceToHost, s);
    cudaError_t ef = cudaFreeAsync(buf, s);
    cudaError_t es = cudaStreamSynchronize(s);
    if (st != PNDF_OK) return st;
    if (e != cudaSuccess || ef != cudaSuccess || es != cudaSuccess) return PNDF_ERR_CUDA;
    return PNDF_OK;
}

pndf_status pndf_diffuse_projected_area(const pndf_hierarchy *h, const pndf_query *q_dev, const float *omega_dev,
                                        int64_t nq, float *P_out_dev, void *stream)
{
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    if (nq < 0 || nq > int64_t(0x7fffffff)) return PNDF_ERR_INVALID_ARG;
    if (nq > 0 && (!q_dev || !omega_dev || !P_out_dev)) return PNDF_ERR_INVALID_ARG;
    if (q_dev && !aligned(q_dev, 16)) return PNDF_ERR_INVALID_ARG;
    return launch_projarea(h, q_dev, omega_dev, nq, P_out_dev, as_stream(stream));
}

pndf_status pndf_shard_work(const pndf_query *q_dev, const uint32_t *order_dev, int64_t nq, int32_t block,
                            double *partial_out_dev, void *stream)
{
    if (nq < 0 || block < 256 || block > (1 << 20)) return PNDF_ERR_INVALID_ARG;
    if (nq == 0) return PNDF_OK;
    if (!q_dev || !order_dev || !partial_out_dev || !aligned(q_dev, 16) || !aligned(order_dev, 4) ||
        !aligned(partial_out_dev, 8))
        return PNDF_ERR_INVALID_ARG;
    return launch_shard_work(q_dev, order_dev, nq, block, partial_out_dev, as_stream(stream)) == cudaSuccess
               ? PNDF_OK
               : PNDF_ERR_CUDA;
}

pndf_status pndf_gather_queries(const pndf_query *q_dev, const uint32_t *order_dev, int64_t first, int64_t count,
                                pndf_query *q_out_dev, void *stream)
{
    if (first < 0 || count < 0) return PNDF_ERR_INVALID_ARG;
    if (count == 0) return PNDF_OK;
    if (!q_dev || !order_dev || !q_out_dev || !aligned(q_dev, 16) || !aligned(order_dev, 4) || !aligned(q_out_dev, 16))
        return PNDF_ERR_INVALID_ARG;
    return launch_gather_queries(q_dev, order_dev, first, count, q_out_dev, as_stream(stream)) == cudaSuccess
               ? PNDF_OK
               : PNDF_ERR_CUDA;
}

pndf_status pndf_scatter_results(const float *D_shard_dev, const uint32_t *order_dev, int64_t first, int64_t count,
                                 float *D_out_dev, void *stream)
{
    if (first < 0 || count < 0) return PNDF_ERR_INVALID_ARG;
    if (count == 0) return PNDF_OK;
    if (!D_shard_dev || !order_dev || !D_out_dev || !aligned(D_shard_dev, 4) || !aligned(order_dev, 4) ||
        !aligned(D_out_dev, 4))
        return PNDF_ERR_INVALID_ARG;
    return launch_scatter_results(D_shard_dev, order_dev, first, count, D_out_dev, as_stream(stream)) == cudaSuccess
               ? PNDF_OK
               : PNDF_ERR_CUDA;
}

pndf_status pndf_device_status(void *stream, uint32_t *bits_out)
{
    std::lock_guard<std::mutex> lock(g_status_mutex);
    unsigned int *host = nullptr, *dev = nullptr;
    cudaError_t e = status_buffer(&host, &dev);
    if (e == cudaSuccess) e = take_status_eval(dev, as_stream(stream));
    if (e == cudaSuccess) e = take_status_projarea(dev + 1, as_stream(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
    const uint32_t bits = e == cudaSuccess ? host[0] | host[1] : 0u;
    if (bits_out) *bits_out = bits;
    if (e != cudaSuccess) return PNDF_ERR_CUDA;
    return bits ? PNDF_ERR_DEVICE : PNDF_OK;
}

pndf_status pndf_last_device_status(const pndf_hierarchy *h, void *stream, uint32_t *bits_out)
{
    if (bits_out) *bits_out = 0;
    pndf_status st = check_hierarchy(h);
    if (st != PNDF_OK) return st;
    std::lock_guard<std::mutex> lock(g_status_mutex);
    unsigned int *host = nullptr, *dev = nullptr;
    cudaError_t e = status_buffer(&host, &dev);
    if (e == cudaSuccess) {
        take_word<<<1, 1, 0, as_stream(stream)>>>(h->d.status, dev + 2);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return PNDF_ERR_CUDA;
    if (bits_out) *bits_out = host[2];
    return host[2] ? PNDF_ERR_DEVICE : PNDF_OK;
}

const char *pndf_status_string(pndf_status s)
{
    switch (s) {
    case PNDF_OK: return "ok";
    case PNDF_ERR_INVALID_ARG: return "invalid argument";
    case PNDF_ERR_OOM: return "out of device memory";
    case PNDF_ERR_CUDA: return "CUDA runtime error";
    case PNDF_ERR_TIMEOUT: return "device wait timed out";
    case PNDF_ERR_CAPACITY: return "device buffer capacity exceeded";
    case PNDF_ERR_UNSUPPORTED: return "unsupported request";
    case PNDF_ERR_DEVICE: return "kernel recorded a device-side error";
    }
    return "unknown status";
}

int32_t pndf_version(void) { return 100; }

int64_t pndf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
