// Min/max normal-bound pyramid build (Sec. 4.2, Fig. 5a).
//
// A node at level l covers 2^l x 2^l quads and stores the bounding box
// (s_min, t_min, s_max, t_max) of the normals of every texel its quads touch,
// so each normal triangle below it lies inside the box.  Levels
// kLeafLevel..L are stored; level l is a (2^(L-l))^2 array in Morton order,
// so the four children of node k at level l are nodes 4k..4k+3 at level l-1
// (one 64-byte line in FP32, one 32-byte sector in FP16).
//
// Level 0 holds one box per quad (its four texels) and, beside it, the
// quad's capsule (the segment between its two farthest normals and a radius
// holding the other two; see common.cuh); the leaf level 2 box is the union
// of its 16 quad boxes.
//
// Kernel 1 (build_tiles): one CTA per 64 x 64-quad tile.  The tile's 65 x 65
// texels are staged in shared memory with 16-byte vector loads (float4 = two
// FP32 texels, uint4 = four FP16 texels) and stored unchanged into the
// hierarchy's own copy of the map (each texel by exactly one tile, so the map
// is read once per build); each thread builds one leaf node's 16 quad boxes
// and their union, and levels up to 6 are reduced in shared memory.  A tile
// is a Morton-aligned square at every level, so its nodes form one contiguous
// run and the writes are fully coalesced.
// Kernel 2 (build_up): one launch per level above the tile, four contiguous
// children reduced per thread.
// FP16 bounds round outward (min toward -inf, max toward +inf) so pruning
// stays conservative: the FP16 box contains the FP32 box.
#include "common.cuh"

namespace pndf {
namespace {

constexpr int kTileQuadsMax = 64;
constexpr int kTileTexMax = kTileQuadsMax + 1;
constexpr int kBuildThreads = 256;


// The quad box as the traversal will read it back (binary16 bounds rounded
// outward, so the decoded box is the stored one).
template <int BFMT>
__device__ __forceinline__ Box stored_box(const Box &b)
{
    if (BFMT == PNDF_BOUNDS_F32) return b;
    return Box{__half2float(__float2half_rd(b.smin)), __half2float(__float2half_rd(b.tmin)),
               __half2float(__float2half_ru(b.smax)), __half2float(__float2half_ru(b.tmax))};
}

// Capsule code of a quad with normals v[0..3] and stored box sb: the segment
// between the farthest pair, as 8-bit fractions of the box; w = the largest
// distance of the four normals to the decoded segment, enlarged by 2^-9
// relative and 2^-21 absolute (more than the FP32 rounding of this distance
// here and of the query's test) and rounded up to binary16.
__device__ __forceinline__ uint2 encode_capsule(const float2 v[4], const Box &sb)
{
    int ip = 0, iq = 1;
    float best = -1.f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i + 1; j < 4; ++j) {
            const float dx = v[j].x - v[i].x, dy = v[j].y - v[i].y;
            const float d2 = fmaf(dx, dx, dy * dy);
            if (d2 > best) {
                best = d2;
                ip = i;
                iq = j;
            }
        }
    auto frac = [](float x, float lo, float hi) -> uint32_t {
        const float e = hi - lo;
        if (!(e > 0.f)) return 0u;
        return uint32_t(fminf(fmaxf(rintf((x - lo) / e * 255.0f), 0.f), 255.f));
    };
    uint2 code;
    code.x = frac(v[ip].x, sb.smin, sb.smax) | (frac(v[ip].y, sb.tmin, sb.tmax) << 8) |
             (frac(v[iq].x, sb.smin, sb.smax) << 16) | (frac(v[iq].y, sb.tmin, sb.tmax) << 24);
    code.y = 0u;
    const Capsule c = decode_capsule(sb.smin, sb.tmin, sb.smax, sb.tmax, code);
    const float L2 = fmaf(c.dx, c.dx, c.dy * c.dy);
    float w = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float ax = v[k].x - c.px, ay = v[k].y - c.py;
        float t = L2 > 0.f ? fminf(fmaxf(fmaf(ax, c.dx, ay * c.dy) / L2, 0.f), 1.f) : 0.f;
        const float ex = fmaf(-t, c.dx, ax), ey = fmaf(-t, c.dy, ay);
        w = fmaxf(w, sqrtf(fmaf(ex, ex, ey * ey)));
    }
    w = fmaf(w, 1.0f + 1.0f / 512.0f, 1.0f / 2097152.0f);
    code.y = uint32_t(__half_as_ushort(__float2half_ru(w)));
    return code;
}

template <int TFMT>
__device__ __forceinline__ float2 load_texel(const void *t, size_t idx)
{
    if (TFMT == PNDF_TEXEL_F32X2) return reinterpret_cast<const float2 *>(t)[idx];
    return __half22float2(reinterpret_cast<const __half2 *>(t)[idx]);
}

// Texel idx of src, loaded for staging and (own) stored unchanged in dst.
template <int TFMT>
__device__ __forceinline__ float2 copy_texel(const void *src, void *dst, size_t idx, bool own)
{
    if (TFMT == PNDF_TEXEL_F32X2) {
        float2 v = reinterpret_cast<const float2 *>(src)[idx];
        if (own) reinterpret_cast<float2 *>(dst)[idx] = v;
        return v;
    }
    __half2 v = reinterpret_cast<const __half2 *>(src)[idx];
    if (own) reinterpret_cast<__half2 *>(dst)[idx] = v;
    return __half22float2(v);
}

// VEC = texels per 16-byte load (2 for FP32, 4 for FP16), or 1 when rows are
// not 16-byte aligned (n not a multiple of VEC).
template <int TFMT, int BFMT, int VEC>
__global__ void __launch_bounds__(kBuildThreads) build_tiles(const void *__restrict__ src, MapDesc d, int tileQ,
                                                            int lq)
{
    __shared__ float2 tex[kTileTexMax * kTileTexMax];
    __shared__ Box box[2][(kTileQuadsMax / kLeafQuads) * (kTileQuadsMax / kLeafQuads)];

    const int n = d.n;
    const int tw = tileQ + 1;
    const int c0 = blockIdx.x * tileQ, r0 = blockIdx.y * tileQ;
    const int tid = threadIdx.x;

    // ---- stage texels: VEC-wide loads for the first tileQ columns.  The
    // hierarchy's own copy of the map is written on the way: a tile owns its
    // first tileQ rows and columns, and the map's last row or column where it
    // is the tile's shared edge, so every texel is stored exactly once ----
    void *copy = const_cast<void *>(d.texels);
    const int nvec = tileQ / VEC;
    for (int idx = tid; idx < tw * nvec; idx += kBuildThreads) {
        int r = idx / nvec, v = idx - r * nvec;
        int gr = r0 + r, gc = c0 + v * VEC;
        if (gr >= n || gc >= n) continue;
        const bool own = r < tileQ || gr == n - 1;
        size_t g = size_t(gr) * n + gc;
        float2 *dst = &tex[r * kTileTexMax + v * VEC];
        if (VEC == 2) {
            float4 p = reinterpret_cast<const float4 *>(src)[g >> 1];
            if (own) reinterpret_cast<float4 *>(copy)[g >> 1] = p;
            dst[0] = make_float2(p.x, p.y);
            dst[1] = make_float2(p.z, p.w);
        } else if (VEC == 4) {
            uint4 p = reinterpret_cast<const uint4 *>(src)[g >> 2];
            if (own) reinterpret_cast<uint4 *>(copy)[g >> 2] = p;
            dst[0] = __half22float2(*reinterpret_cast<__half2 *>(&p.x));
            dst[1] = __half22float2(*reinterpret_cast<__half2 *>(&p.y));
            dst[2] = __half22float2(*reinterpret_cast<__half2 *>(&p.z));
            dst[3] = __half22float2(*reinterpret_cast<__half2 *>(&p.w));
        } else {
            dst[0] = copy_texel<TFMT>(src, copy, g, own);
        }
    }
    // the shared last column of the tile
    for (int r = tid; r < tw; r += kBuildThreads) {
        int gr = r0 + r, gc = c0 + tileQ;
        if (gr < n && gc < n)
            tex[r * kTileTexMax + tileQ] =
                copy_texel<TFMT>(src, copy, size_t(gr) * n + gc, gc == n - 1 && (r < tileQ || gr == n - 1));
    }
    __syncthreads();

    // ---- quads (level 0) and leaf nodes: thread i owns the leaf node with
    // local Morton index i and its 16 quads, whose Morton indices at level 0
    // are 16 i .. 16 i + 15 (a contiguous run of the tile's level-0 block) ----
    const int T = tileQ / kLeafQuads;  // leaf nodes per tile side
    const uint32_t tile_m = morton2(blockIdx.x, blockIdx.y);
    int cur = T * T;
    if (tid < cur) {
        int a = compact1by1(tid), c = compact1by1(tid >> 1);
        Box b = empty_box();
        const size_t qbase = (size_t(tile_m) * cur + tid) * (kLeafQuads * kLeafQuads);
        for (int k = 0; k < kLeafQuads * kLeafQuads; ++k) {
            int lx = a * kLeafQuads + int(compact1by1(k)), ly = c * kLeafQuads + int(compact1by1(k >> 1));
            Box qb = empty_box();
            uint2 cap = make_uint2(0u, 0u);
            if (c0 + lx <= n - 2 && r0 + ly <= n - 2) {
                float2 tv[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float2 t = tex[(ly + (v >> 1)) * kTileTexMax + lx + (v & 1)];
                    tv[v] = t;
                    qb.smin = fminf(qb.smin, t.x);
                    qb.tmin = fminf(qb.tmin, t.y);
                    qb.smax = fmaxf(qb.smax, t.x);
                    qb.tmax = fmaxf(qb.tmax, t.y);
                }
                cap = encode_capsule(tv, stored_box<BFMT>(qb));
            }
            store_box<BFMT>(const_cast<void *>(d.lv[0]), qbase + k, qb);
            const_cast<uint2 *>(d.qcap)[qbase + k] = cap;
            grow(b, qb);
        }
        box[0][tid] = b;
        store_box<BFMT>(const_cast<void *>(d.lv[kLeafLevel]), size_t(tile_m) * cur + tid, b);
    }
    __syncthreads();

    // ---- reduce inside the tile up to level lq ----
    int s = 0;
    for (int l = kLeafLevel + 1; l <= lq; ++l) {
        cur >>= 2;
        if (tid < cur) {
            Box b = box[s][4 * tid];
            grow(b, box[s][4 * tid + 1]);
            grow(b, box[s][4 * tid + 2]);
            grow(b, box[s][4 * tid + 3]);
            box[s ^ 1][tid] = b;
            store_box<BFMT>(const_cast<void *>(d.lv[l]), size_t(tile_m) * cur + tid, b);
        }
        s ^= 1;
        __syncthreads();
    }
}

template <int BFMT>
__global__ void build_up(const void *__restrict__ child, void *__restrict__ parent, size_t count)
{
    size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= count) return;
    Box b = load_box<BFMT>(child, 4 * i);
    grow(b, load_box<BFMT>(child, 4 * i + 1));
    grow(b, load_box<BFMT>(child, 4 * i + 2));
    grow(b, load_box<BFMT>(child, 4 * i + 3));
    if (BFMT == PNDF_BOUNDS_F32) {
        store_box<BFMT>(parent, i, b);
    } else {
        // children are already binary16 values: the reduction is exact
        __half2 lo = __floats2half2_rn(b.smin, b.tmin);
        __half2 hi = __floats2half2_rn(b.smax, b.tmax);
        uint2 v;
        v.x = *reinterpret_cast<uint32_t *>(&lo);
        v.y = *reinterpret_cast<uint32_t *>(&hi);
        reinterpret_cast<uint2 *>(parent)[i] = v;
    }
}

template <int TFMT, int BFMT>
cudaError_t launch_tiles(const void *src, const MapDesc &d, cudaStream_t s)
{
    const int side = 1 << d.L;
    const int tileQ = side < kTileQuadsMax ? side : kTileQuadsMax;
    int lq = 0;
    while ((1 << lq) < tileQ) ++lq;
    dim3 grid(side / tileQ, side / tileQ);
    constexpr int VEC = TFMT == PNDF_TEXEL_F32X2 ? 2 : 4;
    if (d.n % VEC == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0)
        build_tiles<TFMT, BFMT, VEC><<<grid, kBuildThreads, 0, s>>>(src, d, tileQ, lq);
    else
        build_tiles<TFMT, BFMT, 1><<<grid, kBuildThreads, 0, s>>>(src, d, tileQ, lq);
    count_launches(1 + (d.L > lq ? d.L - lq : 0));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int l = lq + 1; l <= d.L; ++l) {
        size_t cnt = level_nodes(d.L, l);
        unsigned blocks = unsigned((cnt + 255) / 256);
        build_up<BFMT><<<blocks, 256, 0, s>>>(d.lv[l - 1], const_cast<void *>(d.lv[l]), cnt);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_build(const void *texels_src, pndf_hierarchy *h, cudaStream_t s)
{
    const MapDesc &d = h->d;
    cudaError_t e;
    if (d.texel_fmt == PNDF_TEXEL_F32X2)
        e = d.bounds_fmt == PNDF_BOUNDS_F32 ? launch_tiles<PNDF_TEXEL_F32X2, PNDF_BOUNDS_F32>(texels_src, d, s)
                                            : launch_tiles<PNDF_TEXEL_F32X2, PNDF_BOUNDS_F16_OUTWARD>(texels_src, d, s);
    else
        e = d.bounds_fmt == PNDF_BOUNDS_F32 ? launch_tiles<PNDF_TEXEL_F16X2, PNDF_BOUNDS_F32>(texels_src, d, s)
                                            : launch_tiles<PNDF_TEXEL_F16X2, PNDF_BOUNDS_F16_OUTWARD>(texels_src, d, s);
    if (e == cudaSuccess && h->clusters) e = launch_clusters(h, s);
    return e;
}

}  // namespace pndf
