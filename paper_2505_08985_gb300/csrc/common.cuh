// Internal definitions shared by the library's CUDA translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pndf.h"

namespace pndf {

constexpr int kMaxLevels = 16;
constexpr int kServeMaxMaps = 8;     // hierarchies per server
constexpr int kLeafLevel = 2;        // stored bottom level: 4 x 4 quads = 32 triangles = one warp
constexpr int kLeafQuads = 1 << kLeafLevel;
constexpr int kLeafTexels = kLeafQuads + 1;
constexpr float kQCut = 16.0f;       // 4-sigma ellipse: d^T S^-1 d <= 16
// Node pruning keeps a relative margin over the cut so that FP32 rounding in
// the box minimum can never prune a node holding a contributing hit.
constexpr float kQPrune = 16.0f * (1.0f + 1e-4f);
constexpr float kTinyCross = 2e-10f; // |cross| below this (area < 1e-10): FP64 triangle test
constexpr float kPi = 3.14159265358979323846f;

// Device view of one hierarchy, passed by value to kernels.
struct MapDesc {
    const void *texels;     // N*N texels (float2 or __half2), row-major
    int n;                  // texels per side
    int L;                  // top level: 2^L >= n - 1 quads per side
    int texel_fmt;          // pndf_texel_fmt
    int bounds_fmt;         // pndf_bounds_fmt
    const void *lv[kMaxLevels];  // level 0 (one box per quad) and levels kLeafLevel..L:
                                 // (2^(L-l))^2 nodes each, Morton order
    unsigned int *status;        // this hierarchy's status word (PNDF_QF_* bits OR-ed in on errors)
    const uint2 *qcap;           // per-quad capsules (level-0 companion, same Morton order)
};

// Record device-side error bits: in the hierarchy's own word and in the
// per-device word of the kernel's translation unit.
__device__ __forceinline__ void record_status(unsigned int *hier_word, unsigned int *device_word, unsigned int bits)
{
    if (hier_word) atomicOr(hier_word, bits);
    atomicOr(device_word, bits);
}

// Cluster hierarchy (Sec. 4.2, Eq. 7-8, App. A), levels kLeafLevel..L in the
// same Morton order as the boxes.  Per node two float4 records,
// (c00.s, c00.t, d10.s, d10.t) and (d01.s, d01.t, d11.s, d11.t) with the
// corner normals c10 = c00 + d10 etc. kept as differences (a flat cluster's
// Jacobian is the cross product of small differences), and the residual e
// (+inf where the node has no cluster).
struct ClusterDesc {
    const float4 *cl[kMaxLevels];
    const float *ce[kMaxLevels];
};

// Morton (Z-order) interleave of two 16-bit coordinates: x in the even bits.
__host__ __device__ __forceinline__ uint32_t part1by1(uint32_t v)
{
    v &= 0x0000ffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t morton2(uint32_t x, uint32_t y)
{
    return part1by1(x) | (part1by1(y) << 1);
}
__host__ __device__ __forceinline__ uint32_t compact1by1(uint32_t v)
{
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}

// Number of levels above the quads: smallest L with 2^L >= n - 1, at least the leaf level.
inline int top_level(int n)
{
    int L = 0;
    while ((1 << L) < n - 1) ++L;
    return L < kLeafLevel ? kLeafLevel : L;
}

// Node box (s_min, t_min, s_max, t_max); empty = (+inf, +inf, -inf, -inf).
// Stored as float4 (FP32 bounds) or as two half2 (FP16 bounds, min rounded
// down and max rounded up).
struct Box {
    float smin, tmin, smax, tmax;
};

__device__ __forceinline__ Box empty_box()
{
    return Box{__int_as_float(0x7f800000), __int_as_float(0x7f800000), __int_as_float(0xff800000),
               __int_as_float(0xff800000)};
}

__device__ __forceinline__ void grow(Box &b, const Box &o)
{
    b.smin = fminf(b.smin, o.smin);
    b.tmin = fminf(b.tmin, o.tmin);
    b.smax = fmaxf(b.smax, o.smax);
    b.tmax = fmaxf(b.tmax, o.tmax);
}

template <int BFMT>
__device__ __forceinline__ void store_box(void *lv, size_t idx, const Box &b)
{
    if (BFMT == PNDF_BOUNDS_F32) {
        reinterpret_cast<float4 *>(lv)[idx] = make_float4(b.smin, b.tmin, b.smax, b.tmax);
    } else {
        __half2 lo = __halves2half2(__float2half_rd(b.smin), __float2half_rd(b.tmin));
        __half2 hi = __halves2half2(__float2half_ru(b.smax), __float2half_ru(b.tmax));
        uint2 v;
        v.x = *reinterpret_cast<uint32_t *>(&lo);
        v.y = *reinterpret_cast<uint32_t *>(&hi);
        reinterpret_cast<uint2 *>(lv)[idx] = v;
    }
}

template <int BFMT>
__device__ __forceinline__ Box load_box(const void *lv, size_t idx)
{
    if (BFMT == PNDF_BOUNDS_F32) {
        float4 v = reinterpret_cast<const float4 *>(lv)[idx];
        return Box{v.x, v.y, v.z, v.w};
    } else {
        uint2 v = reinterpret_cast<const uint2 *>(lv)[idx];
        __half2 lo = *reinterpret_cast<__half2 *>(&v.x);
        __half2 hi = *reinterpret_cast<__half2 *>(&v.y);
        float2 l = __half22float2(lo), h = __half22float2(hi);
        return Box{l.x, l.y, h.x, h.y};
    }
}

// Per-quad capsule, the level-0 companion of the quad boxes.  A quad's two
// normal triangles lie in the convex hull of its four normals, and so within
// distance w of the segment p-q between its two farthest normals (distance to
// a segment is convex, so its maximum over the hull is at a vertex).  For a
// quad straddling two flake cells the triangles are long slivers whose box is
// mostly empty; the capsule is far tighter.  Stored in 8 bytes: p and q as
// 8-bit fractions of the quad's stored box (x: px, py, qx, qy from the low
// byte up), w as binary16 in the low half of y, rounded up with a margin that
// covers FP32 rounding at build and at query time.  Build and query decode
// with this same function, so both see the same segment.
struct Capsule {
    float px, py, dx, dy;  // p and q - p
    float w;
};

__device__ __forceinline__ Capsule decode_capsule(float smin, float tmin, float smax, float tmax, uint2 code)
{
    const float ex = (smax - smin) * (1.0f / 255.0f), ey = (tmax - tmin) * (1.0f / 255.0f);
    Capsule c;
    c.px = fmaf(ex, float(code.x & 255u), smin);
    c.py = fmaf(ey, float((code.x >> 8) & 255u), tmin);
    c.dx = fmaf(ex, float((code.x >> 16) & 255u), smin) - c.px;
    c.dy = fmaf(ey, float(code.x >> 24), tmin) - c.py;
    c.w = __half2float(__ushort_as_half(static_cast<unsigned short>(code.y & 0xffffu)));
    return c;
}

// Distance from (mx, my) to the capsule's segment, squared and compared with
// r^2 without a division: beyond either end the distance to that end,
// between them the perpendicular distance (cross^2 <= r^2 |d|^2).
__device__ __forceinline__ bool capsule_holds(const Capsule &c, float mx, float my, float r)
{
    const float ax = mx - c.px, ay = my - c.py;
    const float t = fmaf(ax, c.dx, ay * c.dy);
    const float L2 = fmaf(c.dx, c.dx, c.dy * c.dy);
    const float r2 = r * r;
    if (t <= 0.f) return fmaf(ax, ax, ay * ay) <= r2;
    if (t >= L2) {
        const float bx = ax - c.dx, by = ay - c.dy;
        return fmaf(bx, bx, by * by) <= r2;
    }
    const float cr = fmaf(ax, c.dy, -ay * c.dx);
    return cr * cr <= r2 * L2;
}

__host__ __device__ inline size_t level_nodes(int L, int l)
{
    size_t s = size_t(1) << (L - l);
    return s * s;
}

}  // namespace pndf

// Opaque hierarchy (host side).
struct pndf_hierarchy {
    int device;
    pndf::MapDesc d;
    void *mem;
    size_t bytes;
    int clusters;              // cluster hierarchy built (and node boxes widened to hold it)
    pndf::ClusterDesc c;       // cluster records, when clusters != 0
    void *moments;             // build scratch: FP64 moments of the level-6 and level-7 nodes
};

namespace pndf {
// launchers implemented in the kernel translation units
cudaError_t launch_build(const void *texels_src, pndf_hierarchy *h, cudaStream_t s);
// Cluster fits of every node and the widened boxes (after launch_build's pyramid).
cudaError_t launch_clusters(pndf_hierarchy *h, cudaStream_t s);
// Bytes of the cluster build scratch for a pyramid of height L.
size_t cluster_scratch_bytes(int L);
// P-NDF sampling (sample.cu).
cudaError_t launch_sample(const pndf_hierarchy *h, const pndf_query *q, const float *u, int64_t n, int kernel,
                          float jac_eps, float *m, uint32_t *tri, uint32_t *flags, cudaStream_t s);
// Level l's cluster records and residuals in row-major node order.
cudaError_t launch_cluster_copy(const pndf_hierarchy *h, int l, float *rec, float *e, cudaStream_t s);
pndf_status launch_eval(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, float *D, uint32_t *flags,
                        pndf_query_stats *stats, const pndf_eval_config &cfg, cudaStream_t s);
pndf_status launch_projarea(const pndf_hierarchy *h, const pndf_query *q, const float *omega, int64_t nq,
                            float *P, cudaStream_t s);
// Evaluation order of a batch (key + counting sort).
pndf_status launch_sort(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, uint32_t *order, cudaStream_t s);
// What a server evaluates for every query (fixed per server).
struct ServeVariant {
    int kernel;     // pndf_kernel
    float tau;      // > 0: the cluster cut (Gaussian only)
    float jac_eps;  // > 0: the Eq. 6 clamp (Gaussian only, tau = 0)
};
// Lets the serving kernel of variant v use the shared memory of `warps` warps
// per CTA; called once before the step graphs are captured.
cudaError_t prepare_serve(int texel_fmt, int bounds_fmt, const ServeVariant &v, int warps);
// One serving step over a device segment table (see serve.cu); clusters:
// per-map cluster descriptors, read only when v.tau > 0.  split: device
// scratch of serve_split_bytes(split_cap) bytes for dividing the step's large
// footprints among warps (null: one warp per query).
cudaError_t launch_serve(int texel_fmt, int bounds_fmt, const ServeVariant &v, const MapDesc *maps,
                         const ClusterDesc *clusters, int nmaps, const uint32_t *table, const pndf_segment *segs,
                         unsigned long long *cursor, int warps, int ctas_per_sm, void *split, uint32_t split_cap,
                         cudaStream_t s);
uint32_t serve_split_cap();
size_t serve_split_bytes(uint32_t cap);
// Allocation-free evaluation with the sort scratch in a fixed device array.
pndf_status launch_eval_noalloc(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, float *D, uint32_t *flags,
                                cudaStream_t s);
int64_t noalloc_max_queries();
// Count of kernels launched by the library (host-side, process-wide).
void count_launches(int64_t n);
// Each kernel translation unit keeps its own device status word (PNDF_QF_*
// bits OR-ed in by kernels on errors).  These queue, on s, a kernel that
// takes the word (atomic exchange with 0, so bits OR-ed in concurrently are
// never lost) and stores the old value at out (page-locked host memory).
cudaError_t take_status_eval(unsigned int *out, cudaStream_t s);
cudaError_t take_status_projarea(unsigned int *out, cudaStream_t s);
}  // namespace pndf
