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

inline size_t level_nodes(int L, int l)
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
};

namespace pndf {
// launchers implemented in the kernel translation units
cudaError_t launch_build(const void *texels_src, pndf_hierarchy *h, cudaStream_t s);
pndf_status launch_eval(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, float *D, uint32_t *flags,
                        pndf_query_stats *stats, const pndf_eval_config &cfg, cudaStream_t s);
pndf_status launch_projarea(const pndf_hierarchy *h, const pndf_query *q, const float *omega, int64_t nq,
                            float *P, cudaStream_t s);
// Evaluation order of a batch (key + counting sort).
pndf_status launch_sort(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, uint32_t *order, cudaStream_t s);
// One serving step over a device segment table (see serve.cu).
cudaError_t launch_serve(int texel_fmt, int bounds_fmt, const MapDesc *maps, int nmaps, const uint32_t *table,
                         const pndf_segment *segs, unsigned long long *cursor, int warps, int ctas_per_sm,
                         cudaStream_t s);
// Allocation-free evaluation with the sort scratch in a fixed device array.
pndf_status launch_eval_noalloc(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, float *D, uint32_t *flags,
                                cudaStream_t s);
int64_t noalloc_max_queries();
// Count of kernels launched by the library (host-side, process-wide).
void count_launches(int64_t n);
// Each kernel translation unit keeps its own device status word (PNDF_QF_*
// bits OR-ed in by kernels on errors); these read it and optionally clear it.
cudaError_t read_status_eval(cudaStream_t s, uint32_t *bits, bool clear);
cudaError_t read_status_projarea(cudaStream_t s, uint32_t *bits, bool clear);
}  // namespace pndf
