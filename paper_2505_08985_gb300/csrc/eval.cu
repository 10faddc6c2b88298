// Batched P-NDF evaluation over the position-normal manifold (Sec. 4.1-4.2).
//
// Per query (footprint centre x, covariance S, normal m) the result is Eq. 5:
//   D = sum over triangles abc with m in n(abc) of
//       k_r(a l0 + b l1 + c l2 - x) / |(n_b - n_a) x (n_c - n_a)|.
//
// Pipeline (all on the caller's stream):
//   key_hist  : per query a key of 4 + sub bits: the entry level (App. C; the
//               smallest level whose node side reaches the support's
//               half-width), largest footprints first, above a sub-key of 6..14
//               bits (footprint tile and/or query-normal bin); counted into a
//               global histogram with atomics.
//   key_scan  : exclusive scan of the histogram (one CTA).
//   key_place : counting-sort placement -> query order.
//   traverse  : persistent warps pull queries from an atomic cursor; one warp
//               per query.  Depth-first descent of the min/max pyramid with a
//               per-warp shared-memory stack: each step pops up to 16 nodes,
//               lane k tests child (k & 3) of popped nodes (k >> 2) and
//               (k >> 2) + 8 - uv box against the support first, then the
//               normal box against m - and ballot/popc compaction pushes the
//               survivors.  Surviving leaf blocks (4 x 4 quads) have their 16
//               per-quad boxes (level 0, one 128-byte line in FP16) tested four
//               per lane in one load, eight blocks per pass; quads whose box
//               holds m are compacted into a per-warp ring and taken 64 at a
//               time (two per lane, both loads in flight) through the quad's
//               capsule (segment between its farthest normals plus a radius,
//               the tight bound for slivers across normal discontinuities);
//               capsule survivors are compacted again and tested 32 at a
//               time (lane = quad, both triangles), and edge-test hits are
//               compacted once more and weighed 32 at a time.  Each weight
//               is added exactly into the thread's 128-bit fixed-point sum;
//               the warp's sums are added exactly and the total is written in
//               caller order (the unpermute is fused into the store).  Large
//               footprints of a batch are divided into tiles of nodes, one
//               warp per tile (split_work / split_plan).  Flat mode skips
//               every box and tests all 32 triangles of every leaf block in
//               the support's bounding box.
// Hit test (tie rule): m inside the closed normal bounding box and all three
// edge functions sign-consistent with the triangle orientation (>= 0 after
// orientation, i.e. closed barycentrics).  Zero-area normal triangles are a
// delta and are skipped.  Edge functions use an FMA difference of products on
// vertex-relative differences; triangles whose FP32 |cross| is below 2e-10
// (normal-space area below 1e-10) are re-tested and weighted in FP64.
#include <mutex>

#include "common.cuh"

namespace pndf {

__device__ unsigned int g_status_eval;

namespace {

constexpr int kStackCap = 768;     // DFS stack entries per warp (about 48 per level + 64 in the worst case)
constexpr int kMaxSubBits = 14;                   // sub-key bits below the 4 entry-level bits
constexpr int kKeyBins = 1 << (4 + kMaxSubBits);  // largest histogram (2^18 bins)
#ifndef PNDF_TRAVERSE_MIN_CTAS
// 3 x 256 threads per SM at <= 85 registers: with two capsule tests per lane
// in flight this measured 916 ms per 4M-query flake step, against 1008 ms at
// 4 CTAs (64 registers, more spills) and 1154 ms at 2
#define PNDF_TRAVERSE_MIN_CTAS 3
#endif
constexpr unsigned kFull = 0xffffffffu;

// Kahan's difference of products a*b - c*d with one FMA correction.
__device__ __forceinline__ float dop(float a, float b, float c, float d)
{
    float w = c * d;
    float e = fmaf(-c, d, w);
    float f = fmaf(a, b, -w);
    return f + e;
}

// Twice the signed area of (p, q, r): (q - p) x (r - p).
__device__ __forceinline__ float orient(float px, float py, float qx, float qy, float rx, float ry)
{
    return dop(qx - px, ry - py, qy - py, rx - px);
}

__device__ __forceinline__ double orient_d(double px, double py, double qx, double qy, double rx, double ry)
{
    return (qx - px) * (ry - py) - (qy - py) * (rx - px);
}

// MurmurHash3 32-bit finalizer (Appleby), fingerprints hit sets in stats mode.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Footprint kernels (pndf_kernel): the Gaussian cut at q = d^T S^-1 d <= 16,
// and the disk (q <= 1.5^2) and box (|L^-1 d|_inf <= 1.5, S = L L^T) filters
// of the (3 sigma)^2 footprints the paper pairs with it.
struct Query {
    float x, y;          // footprint centre
    float ia, ib, ic;    // S^-1 = [[ia, ib], [ib, ic]]
    float norm;          // kernel normalisation: 1 / (2 pi, 2.25 pi or 9) sqrt(det S)
    float mx, my;        // query normal
    float rx, ry;        // half-widths of the support's bounding box (slightly inflated)
    float qprune;        // the support lies in q <= qprune (16, 2.25, 4.5), with a margin
    float theta;         // r_x r_y of the support (exact half-widths); times tau for the cluster cut
    float kyx, kxy;      // -ib / ic and -ib / ia: the minimiser of q along a vertical / horizontal line
    float inv_sxx;       // box: 1 / S_xx, so that (L^-1 d)_x^2 = dx^2 / S_xx
    float l11, l21, l22; // box: the Cholesky factor L of S (node tests by separating axes)
    float jac, rho;      // Eq. 6 clamp: Jacobian floor eps and the replacement's circumradius (0: off)
    int kernel;
    bool valid;
};

// Internal kernel id of the Gaussian with the Jacobian clamp of Eq. 6.
constexpr int kKernGaussClamp = 3;

__device__ __forceinline__ Query make_query(const pndf_query &r, int kernel = PNDF_KERNEL_GAUSS, float jac_eps = 0.f)
{
    Query q;
    q.jac = q.rho = 0.f;
    if (kernel == kKernGaussClamp) {
        // equilateral replacement of area eps / 2: side^2 = 2 eps / sqrt(3), circumradius side / sqrt(3)
        q.jac = jac_eps;
        q.rho = sqrtf(2.0f * jac_eps / 1.7320508f) * 0.57735027f;
        kernel = PNDF_KERNEL_GAUSS;
    }
    q.x = r.x;
    q.y = r.y;
    q.mx = r.ms;
    q.my = r.mt;
    q.kernel = kernel;
    float det = r.sxx * r.syy - r.sxy * r.sxy;
    q.valid = (r.sxx > 0.f) && (r.syy > 0.f) && (det > 0.f) && isfinite(det) && isfinite(r.x) &&
              isfinite(r.y) && isfinite(r.ms) && isfinite(r.mt);
    float inv = 1.0f / det;
    q.ia = r.syy * inv;
    q.ib = -r.sxy * inv;
    q.ic = r.sxx * inv;
    q.kyx = -q.ib / q.ic;
    q.kxy = -q.ib / q.ia;
    const float sx = sqrtf(r.sxx), sy = sqrtf(r.syy), sd = sqrtf(det);
    float hx, hy;
    q.inv_sxx = 0.f;
    q.l11 = q.l21 = q.l22 = 0.f;
    if (kernel == PNDF_KERNEL_DISK) {
        q.norm = 1.0f / (2.25f * kPi * sd);
        hx = 1.5f * sx;
        hy = 1.5f * sy;
        q.qprune = 2.25f * (1.0f + 1e-4f);
    } else if (kernel == PNDF_KERNEL_BOX) {
        q.norm = 1.0f / (9.0f * sd);
        const float l21 = r.sxy / sx, l22 = sqrtf(fmaxf(r.syy - l21 * l21, 0.f));
        hx = 1.5f * sx;
        hy = 1.5f * (fabsf(l21) + l22);
        q.qprune = 4.5f * (1.0f + 1e-4f);  // |v|_inf <= 1.5 implies |v|^2 <= 4.5
        q.inv_sxx = 1.0f / r.sxx;
        q.l11 = sx;
        q.l21 = l21;
        q.l22 = l22;
    } else {
        q.norm = 1.0f / (2.0f * kPi * sd);
        hx = 4.0f * sx;  // q <= 16 implies |dx| <= 4 sqrt(sxx)
        hy = 4.0f * sy;
        q.qprune = kQPrune;
    }
    q.theta = hx * hy;
    // inflate so rounding never clips the support's box
    q.rx = hx * (1.0f + 1e-5f) + 1e-6f;
    q.ry = hy * (1.0f + 1e-5f) + 1e-6f;
    return q;
}

// Kernel weight at offset d with q = d^T S^-1 d; 0 outside the support.
__device__ __forceinline__ float kweight(const Query &q, float dx, float qq)
{
    if (q.kernel == PNDF_KERNEL_GAUSS) return qq <= kQCut ? q.norm * expf(-0.5f * qq) : 0.f;
    if (q.kernel == PNDF_KERNEL_DISK) return qq <= 2.25f ? q.norm : 0.f;
    const float v1 = dx * dx * q.inv_sxx;  // (L^-1 d)_x^2; (L^-1 d)_y^2 = q - v1
    return (v1 <= 2.25f && qq - v1 <= 2.25f) ? q.norm : 0.f;
}

__device__ __forceinline__ double kweight_d(const Query &q, double dx, double qq)
{
    if (q.kernel == PNDF_KERNEL_GAUSS) return qq <= double(kQCut) ? double(q.norm) * exp(-0.5 * qq) : 0.0;
    if (q.kernel == PNDF_KERNEL_DISK) return qq <= 2.25 ? double(q.norm) : 0.0;
    const double v1 = dx * dx * double(q.inv_sxx);
    return (v1 <= 2.25 && qq - v1 <= 2.25) ? double(q.norm) : 0.0;
}

__device__ __forceinline__ float qform(const Query &q, float dx, float dy)
{
    return fmaf(q.ia * dx, dx, fmaf(2.0f * q.ib * dx, dy, q.ic * dy * dy));
}

// Minimum of q over the box [dx0, dx1] x [dy0, dy1] (offsets from the centre).
// The quadratic is convex with its minimum at the origin; off the box, the
// minimum lies on an edge whose outer side holds the origin, where it is a
// clamped 1D minimum (along x = X at y = -(ib / ic) X, the ratio precomputed
// per query; a minimiser off by rounding raises the value only to second
// order, far inside the pruning margin).
__device__ __forceinline__ float qmin_box(const Query &q, float dx0, float dx1, float dy0, float dy1)
{
    if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return 0.f;
    float best = __int_as_float(0x7f800000);
    if (dx0 > 0.f || dx1 < 0.f) {
        float X = dx0 > 0.f ? dx0 : dx1;
        float y = fminf(fmaxf(q.kyx * X, dy0), dy1);
        best = fminf(best, qform(q, X, y));
    }
    if (dy0 > 0.f || dy1 < 0.f) {
        float Y = dy0 > 0.f ? dy0 : dy1;
        float x = fminf(fmaxf(q.kxy * Y, dx0), dx1);
        best = fminf(best, qform(q, x, Y));
    }
    return best;
}

// A node's normal box as stored: FP32 (s_min, t_min, s_max, t_max) in x..w,
// or binary16 (s_min, t_min) and (s_max, t_max) as two half2 in x and y
// (decoded only where tested, so a box in flight holds two registers).
template <int BFMT>
__device__ __forceinline__ uint4 node_box(const MapDesc &d, int l, uint32_t m)
{
    if (BFMT == PNDF_BOUNDS_F32) return __ldg(reinterpret_cast<const uint4 *>(d.lv[l]) + m);
    uint2 v = __ldg(reinterpret_cast<const uint2 *>(d.lv[l]) + m);
    return make_uint4(v.x, v.y, 0u, 0u);
}

template <int TFMT>
__device__ __forceinline__ float2 texel(const MapDesc &d, int i, int j)
{
    size_t idx = size_t(j) * d.n + i;
    if (TFMT == PNDF_TEXEL_F32X2) return __ldg(reinterpret_cast<const float2 *>(d.texels) + idx);
    __half2 h = __ldg(reinterpret_cast<const __half2 *>(d.texels) + idx);
    return __half22float2(h);
}

// Box kernel: does [dx0, dx1] x [dy0, dy1] (offsets from the centre) meet the
// support L [-1.5, 1.5]^2?  Separating axes: x and y (the support's extents
// are the inflated half-widths rx, ry) and n = (-l21, l11), normal to L e1,
// onto which the support projects to +-1.5 l11 l22 (slightly inflated).
__device__ __forceinline__ bool box_support_meets(const Query &q, float dx0, float dx1, float dy0, float dy1)
{
    if (dx0 > q.rx || dx1 < -q.rx || dy0 > q.ry || dy1 < -q.ry) return false;
    const float hn = 1.5f * q.l11 * q.l22 * (1.0f + 1e-4f) + 1e-6f;
    const float p0 = -q.l21 * dx0, p1 = -q.l21 * dx1;
    const float pmin = fminf(p0, p1) + q.l11 * dy0, pmax = fmaxf(p0, p1) + q.l11 * dy1;
    return pmin <= hn && pmax >= -hn;
}

// Node (level l, coords a, c): uv box [a 2^l, (a+1) 2^l] x [c 2^l, (c+1) 2^l].
// It can hold a contributing hit only if that box meets the kernel's support
// (the ellipse q <= qprune; for the box kernel the sheared square itself).
__device__ __forceinline__ bool node_in_footprint(const Query &q, int l, uint32_t a, uint32_t c)
{
    float sz = float(1u << l);
    float dx0 = float(a) * sz - q.x, dy0 = float(c) * sz - q.y;
    if (q.kernel == PNDF_KERNEL_BOX) return box_support_meets(q, dx0, dx0 + sz, dy0, dy0 + sz);
    return qmin_box(q, dx0, dx0 + sz, dy0, dy0 + sz) <= q.qprune;
}

// The node's uv box lies entirely inside the pruning region (the quadratic is
// convex, so its maximum over the box is at a corner; the box kernel's
// support is convex too); every descendant then passes the footprint test
// and skips it.  Claiming "inside" wrongly would only prune less.
__device__ __forceinline__ bool node_inside(const Query &q, int l, uint32_t a, uint32_t c)
{
    float sz = float(1u << l);
    float dx0 = float(a) * sz - q.x, dy0 = float(c) * sz - q.y;
    float dx1 = dx0 + sz, dy1 = dy0 + sz;
    if (q.kernel == PNDF_KERNEL_BOX) {  // the support is convex: all four corners inside it
        const float hx = 1.5f * q.l11, hv = 1.5f * q.l22, k = q.l21 / q.l11;
        return fmaxf(fabsf(dx0), fabsf(dx1)) <= hx && fabsf(dy0 - k * dx0) <= hv && fabsf(dy0 - k * dx1) <= hv &&
               fabsf(dy1 - k * dx0) <= hv && fabsf(dy1 - k * dx1) <= hv;
    }
    float m = fmaxf(fmaxf(qform(q, dx0, dy0), qform(q, dx1, dy0)), fmaxf(qform(q, dx0, dy1), qform(q, dx1, dy1)));
    return m <= q.qprune;
}

// m in the box; with the clamp (CLAMP) widened by the replacement radius (a
// replacement lies within rho of its triangle's centroid, hence of its box).
template <bool CLAMP>
__device__ __forceinline__ bool box_holds(const float4 &b, const Query &q)
{
    if (CLAMP) return q.mx >= b.x - q.rho && q.mx <= b.z + q.rho && q.my >= b.y - q.rho && q.my <= b.w + q.rho;
    return q.mx >= b.x && q.mx <= b.z && q.my >= b.y && q.my <= b.w;
}

// m in a node box as stored (node_box).
template <int BFMT, bool CLAMP>
__device__ __forceinline__ bool stored_box_holds(const uint4 &v, const Query &q)
{
    if (BFMT == PNDF_BOUNDS_F32)
        return box_holds<CLAMP>(make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                                            __uint_as_float(v.w)), q);
    float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    return box_holds<CLAMP>(make_float4(lo.x, lo.y, hi.x, hi.y), q);
}

template <int BFMT, bool CLAMP>
__device__ __forceinline__ bool node_test(const MapDesc &d, const Query &q, int l, uint32_t a, uint32_t c)
{
    if (!node_in_footprint(q, l, a, c)) return false;
    return stored_box_holds<BFMT, CLAMP>(node_box<BFMT>(d, l, morton2(a, c)), q);
}

// Stack / leaf-queue entry: level in bits 28-31, "inside the ellipse" in bit
// 27, the node's Morton index at its level in bits 0-26 (at most 2 (L - 1) =
// 26 bits for L <= 14).  A child's Morton index is (m << 2) | (dy << 1 | dx).
__device__ __forceinline__ uint32_t pack(int l, bool inside, uint32_t m)
{
    return (uint32_t(l) << 28) | (uint32_t(inside) << 27) | m;
}
constexpr uint32_t kMortonMask = (1u << 27) - 1u;

// A query's sum is exact: every contribution (an FP32 value >= 0) is added
// into a 128-bit fixed-point number with 64 fraction bits, value =
// (hi 2^64 + lo) 2^-64, so the result does not depend on the order in which
// the hits are found or on how the query's work is divided among warps.  A
// contribution is rounded to the nearest multiple of 2^-64 (5.4e-20) once;
// the total is rounded to FP32 once at the end.  A contribution of 2^63 or
// more, or a sum past 2^64 (only possible for normal triangles of area far
// below 1e-20), marks the query kHuge and its D is +inf.
// The sum lives in shared memory (one 128-bit slot per thread of the CTA,
// at most 256 threads), so the descent keeps its registers; the counters and
// flags stay in registers.
struct Acc {
    uint32_t hits, hash, tests, fp64, degen, leaves, nodes, quads, cchecks, clusters;
    uint32_t flags;
};
constexpr uint32_t kHuge = 1u << 30;  // internal flag bit: the sum is out of the fixed-point range
__shared__ unsigned long long s_sum_lo[256], s_sum_hi[256];

__device__ __forceinline__ void acc_zero()
{
    s_sum_lo[threadIdx.x] = 0ull;
    s_sum_hi[threadIdx.x] = 0ull;
}

__device__ __forceinline__ void acc_add(Acc &a, float w)
{
    const uint32_t b = __float_as_uint(w);
    const int ex = int(b >> 23);  // sign 0: the biased exponent
    if (ex == 0 || (b >> 31)) return;  // zero or subnormal (< 2^-126: rounds to 0)
    if (ex >= 127 + 63) {              // 2^63 or more, inf or NaN
        a.flags |= kHuge;
        return;
    }
    const unsigned long long m = (b & 0x7fffffu) | 0x800000u;  // w = m 2^(ex - 150)
    const int sh = ex - 150 + 64;                               // w 2^64 = m 2^sh
    unsigned long long dl, dh = 0ull;
    if (sh < 0) {
        if (sh < -24) return;                        // below 2^-65: rounds to 0
        dl = (m + (1ull << (-sh - 1))) >> (-sh);     // round half up
    } else if (sh < 64) {
        dl = m << sh;
        if (sh > 40) dh = m >> (64 - sh);
    } else {
        dl = 0ull;
        dh = m << (sh - 64);  // sh <= 189 - 86: dh < 2^63
    }
    const unsigned long long lo = s_sum_lo[threadIdx.x] + dl;
    s_sum_lo[threadIdx.x] = lo;
    const unsigned long long h0 = s_sum_hi[threadIdx.x];
    const unsigned long long hi = h0 + dh + (lo < dl ? 1ull : 0ull);
    s_sum_hi[threadIdx.x] = hi;
    if (hi < h0) a.flags |= kHuge;  // past 2^64
}

// 128-bit fixed point -> FP32 (through FP64: deterministic, within an ulp).
__device__ __forceinline__ float acc_value(unsigned long long lo, unsigned long long hi, uint32_t flags)
{
    if (flags & kHuge) return __int_as_float(0x7f800000);
    return float(double(hi) + double(lo) * 0x1p-64);
}

// Test the lane's triangle of a leaf block and accumulate its contribution.
// tri 0: (u0, u1, u2) with a = (i, j), b = a + (1, 0), c = a + (0, 1);
// tri 1: (u3, u2, u1) with a = (i+1, j+1), b = a - (1, 0), c = a - (0, 1).
template <bool STATS>
__device__ __forceinline__ void test_triangle(const Query &q, float2 na, float2 nb, float2 nc, int ai, int aj,
                                              float dir, uint32_t tri_id, Acc &acc)
{
    if (STATS) acc.tests++;
    float lox = fminf(na.x, fminf(nb.x, nc.x)), hix = fmaxf(na.x, fmaxf(nb.x, nc.x));
    float loy = fminf(na.y, fminf(nb.y, nc.y)), hiy = fmaxf(na.y, fmaxf(nb.y, nc.y));
    if (q.mx < lox || q.mx > hix || q.my < loy || q.my > hiy) return;
    float cr = orient(na.x, na.y, nb.x, nb.y, nc.x, nc.y);
    float l1, l2, J;
    if (fabsf(cr) >= kTinyCross) {
        float e0 = orient(nb.x, nb.y, nc.x, nc.y, q.mx, q.my);
        float e1 = orient(nc.x, nc.y, na.x, na.y, q.mx, q.my);
        float e2 = orient(na.x, na.y, nb.x, nb.y, q.mx, q.my);
        bool hit = cr > 0.f ? (e0 >= 0.f && e1 >= 0.f && e2 >= 0.f) : (e0 <= 0.f && e1 <= 0.f && e2 <= 0.f);
        if (!hit) return;
        float inv = 1.0f / cr;
        l1 = e1 * inv;
        l2 = e2 * inv;
        J = fabsf(cr);
    } else {
        // near-singular normal triangle: FP64 test and weight
        double ax = na.x, ay = na.y, bx = nb.x, by = nb.y, cx = nc.x, cy = nc.y, mx = q.mx, my = q.my;
        double dcr = orient_d(ax, ay, bx, by, cx, cy);
        if (dcr == 0.0) {
            if (STATS) acc.degen++;
            return;
        }
        if (STATS) acc.fp64++;
        acc.flags |= PNDF_QF_FP64;
        double e0 = orient_d(bx, by, cx, cy, mx, my);
        double e1 = orient_d(cx, cy, ax, ay, mx, my);
        double e2 = orient_d(ax, ay, bx, by, mx, my);
        bool hit = dcr > 0.0 ? (e0 >= 0.0 && e1 >= 0.0 && e2 >= 0.0) : (e0 <= 0.0 && e1 <= 0.0 && e2 <= 0.0);
        if (!hit) return;
        double dl1 = e1 / dcr, dl2 = e2 / dcr;
        double dx = (double(ai) - double(q.x)) + dir * dl1;
        double dy = (double(aj) - double(q.y)) + dir * dl2;
        double qq = double(q.ia) * dx * dx + 2.0 * double(q.ib) * dx * dy + double(q.ic) * dy * dy;
        double w = kweight_d(q, dx, qq);
        if (w == 0.0) return;
        w /= fabs(dcr);
        acc_add(acc, float(w));
        if (STATS) {
            acc.hits++;
            acc.hash += fmix32(tri_id);
        }
        return;
    }
    float dx = (float(ai) - q.x) + dir * l1;
    float dy = (float(aj) - q.y) + dir * l2;
    float qq = qform(q, dx, dy);
    float w = kweight(q, dx, qq);
    if (w == 0.f) return;
    acc_add(acc, w / J);
    if (STATS) {
        acc.hits++;
        acc.hash += fmix32(tri_id);
    }
}

// The hit decision of test_triangle alone: true for an FP32 hit (writes the
// orientation-signed cross and edge functions e1, e2, so l1 = e1 / cross,
// l2 = e2 / cross).  Near-singular triangles (FP32 |cross| < 2e-10) are
// decided, weighted and accumulated here in FP64 and return false.
template <bool STATS, bool CLAMP>
__device__ __forceinline__ bool edge_test(const Query &q, float2 na, float2 nb, float2 nc, int ai, int aj, float dir,
                                          uint32_t tri_id, Acc &acc, float &cr_o, float &e1_o, float &e2_o)
{
    if (STATS) acc.tests++;
    float lox = fminf(na.x, fminf(nb.x, nc.x)), hix = fmaxf(na.x, fmaxf(nb.x, nc.x));
    float loy = fminf(na.y, fminf(nb.y, nc.y)), hiy = fmaxf(na.y, fmaxf(nb.y, nc.y));
    if (CLAMP) {
        lox -= q.rho;
        hix += q.rho;
        loy -= q.rho;
        hiy += q.rho;
    }
    if (q.mx < lox || q.mx > hix || q.my < loy || q.my > hiy) return false;
    float cr = orient(na.x, na.y, nb.x, nb.y, nc.x, nc.y);
    if (CLAMP && fabsf(cr) < q.jac) {
        // Eq. 6: the equilateral replacement (vertex k at 90 + 120 k degrees
        // around the centroid g, radius rho), in vertex-relative form p = m - E0
        const float gx = (na.x + nb.x + nc.x) * (1.0f / 3.0f), gy = (na.y + nb.y + nc.y) * (1.0f / 3.0f);
        const float h = 0.8660254f * q.rho;  // E1 - E0 = rho (-sqrt3/2, -3/2), E2 - E0 = rho (sqrt3/2, -3/2)
        const float2 b = make_float2(-h, -1.5f * q.rho), c = make_float2(h, -1.5f * q.rho);
        const float2 p = make_float2(q.mx - gx, (q.my - gy) - q.rho);
        const float ecr = dop(b.x, c.y, b.y, c.x);
        const float e0 = dop(c.x - b.x, p.y - b.y, c.y - b.y, p.x - b.x);
        const float e1 = dop(p.x, c.y, p.y, c.x);
        const float e2 = dop(b.x, p.y, b.y, p.x);
        cr_o = ecr;  // > 0: counter-clockwise
        e1_o = e1;
        e2_o = e2;
        return e0 >= 0.f && e1 >= 0.f && e2 >= 0.f;
    }
    if (fabsf(cr) >= kTinyCross) {
        float e0 = orient(nb.x, nb.y, nc.x, nc.y, q.mx, q.my);
        float e1 = orient(nc.x, nc.y, na.x, na.y, q.mx, q.my);
        float e2 = orient(na.x, na.y, nb.x, nb.y, q.mx, q.my);
        bool hit = cr > 0.f ? (e0 >= 0.f && e1 >= 0.f && e2 >= 0.f) : (e0 <= 0.f && e1 <= 0.f && e2 <= 0.f);
        cr_o = cr;
        e1_o = e1;
        e2_o = e2;
        return hit;
    }
    test_triangle<STATS>(q, na, nb, nc, ai, aj, dir, tri_id, acc);  // FP64 branch
    if (STATS) acc.tests--;
    return false;
}

// Hit ring: FP32 hits waiting for their footprint weight, as (cross, e1, e2,
// tag): tag (i << 15) | (j << 1) | tri for a triangle of quad (i, j), or
// kClusterTag | (l << 27) | (morton << 1) | tri for a cluster triangle of
// node (l, morton).
constexpr int kHitRing = 64;
constexpr uint32_t kClusterTag = 0x80000000u;
constexpr uint32_t kClusterMorton = (1u << 26) - 1u;

// All 32 lanes: lane k < cnt weighs hit k of the ring (the tail of test_triangle).
template <bool STATS>
__device__ __forceinline__ void drain_hits(const Query &q, int n, int L, const float4 *hits, uint32_t hh, int cnt,
                                           int lane, Acc &acc)
{
    if (lane < cnt) {
        float4 h = hits[(hh + uint32_t(lane)) & (kHitRing - 1)];
        uint32_t pk = __float_as_uint(h.w);
        const int tri = int(pk & 1u);
        int gi, gj, l = 0;
        if (pk & kClusterTag) {  // cluster triangle of node (l, I, J): uv scale 2^l
            l = int((pk >> 27) & 15u);
            uint32_t m = (pk >> 1) & kClusterMorton;
            gi = int(compact1by1(m)) << l;
            gj = int(compact1by1(m >> 1)) << l;
        } else {
            gi = int(pk >> 15);
            gj = int((pk >> 1) & 0x3fffu);
        }
        const float a = float(1 << l);
        float inv = 1.0f / h.x;
        float l1 = h.y * inv, l2 = h.z * inv;
        float dir = tri ? -a : a;
        float dx = (float(gi + (tri << l)) - q.x) + dir * l1;
        float dy = (float(gj + (tri << l)) - q.y) + dir * l2;
        float qq = qform(q, dx, dy);
        const float w = kweight(q, dx, qq);
        if (w != 0.f) {
            acc_add(acc, w * (a * a) / fabsf(h.x));
            if (STATS) {
                acc.hits++;
                uint32_t id;
                if (pk & kClusterTag) {
                    uint32_t S = 1u << (L - l);
                    id = kClusterTag | (uint32_t(l) << 27) |
                         (((uint32_t(gj) >> l) * S + (uint32_t(gi) >> l)) << 1) | uint32_t(tri);
                } else {
                    id = 2u * (uint32_t(gj) * uint32_t(n - 1) + uint32_t(gi)) + uint32_t(tri);
                }
                acc.hash += fmix32(id);
            }
        }
    }
}

// Lanes 0..24 fetch the 5 x 5 texels of leaf block (a, c) (4 x 4 quads).
template <int TFMT>
__device__ __forceinline__ float2 leaf_texel(const MapDesc &d, uint32_t a, uint32_t c, int lane)
{
    const int i0 = int(a) << kLeafLevel, j0 = int(c) << kLeafLevel;
    int tc = lane % kLeafTexels, tr = lane / kLeafTexels;
    float2 tv = make_float2(0.f, 0.f);
    if (lane < kLeafTexels * kLeafTexels && i0 + tc < d.n && j0 + tr < d.n) tv = texel<TFMT>(d, i0 + tc, j0 + tr);
    return tv;
}

// All 32 lanes: test the 32 triangles of leaf block (a, c) whose texels the
// lanes hold in tv (lane t: quad t >> 1, triangle t & 1).
template <bool STATS>
__device__ __forceinline__ void test_leaf(const MapDesc &d, const Query &q, uint32_t a, uint32_t c, float2 tv,
                                          int lane, Acc &acc)
{
    const int n = d.n;
    const int i0 = int(a) << kLeafLevel, j0 = int(c) << kLeafLevel;
    int qd = lane >> 1, qx = qd & 3, qy = qd >> 2, tri = lane & 1;
    int base = qy * kLeafTexels + qx;
    int sa = tri ? base + kLeafTexels + 1 : base;
    int sb = tri ? base + kLeafTexels : base + 1;
    int sc = tri ? base + 1 : base + kLeafTexels;
    float2 na, nb, nc;
    na.x = __shfl_sync(kFull, tv.x, sa);
    na.y = __shfl_sync(kFull, tv.y, sa);
    nb.x = __shfl_sync(kFull, tv.x, sb);
    nb.y = __shfl_sync(kFull, tv.y, sb);
    nc.x = __shfl_sync(kFull, tv.x, sc);
    nc.y = __shfl_sync(kFull, tv.y, sc);
    int gi = i0 + qx, gj = j0 + qy;
    if (STATS && lane == 0) acc.leaves++;
    if (gi <= n - 2 && gj <= n - 2) {
        uint32_t id = 2u * (uint32_t(gj) * uint32_t(n - 1) + uint32_t(gi)) + uint32_t(tri);
        test_triangle<STATS>(q, na, nb, nc, tri ? gi + 1 : gi, tri ? gj + 1 : gj, tri ? -1.f : 1.f, id, acc);
    }
}

// Survivor ring: quads whose level-0 box holds m, packed (i << 16) | j.
constexpr int kRing = 256;
// Capsule ring: box survivors whose capsule holds m too (at most 31 held
// over between rounds plus one round's 32).
constexpr int kCapRing = 64;
// Leaf queue: up to 7 leaf blocks held over from the last step plus one
// step's 64 children; cut cluster nodes fill it from the back (entry k at
// kLeafQ - 1 - k), and a step's new leaf blocks and cut nodes number at most
// 64 together, so the two ends never meet.
constexpr int kLeafQ = 72;
// Shared memory per warp: DFS stack, leaf queue, survivor ring, capsule
// ring, hit ring (a multiple of four words, so the hit ring stays 16-byte
// aligned).
constexpr int kWarpSmemWords = kStackCap + kLeafQ + kRing + kCapRing + 4 * kHitRing;
static_assert((kStackCap + kLeafQ + kRing + kCapRing) % 4 == 0, "hit ring alignment");

// Per-warp leaf state: box-survivor ring, capsule-survivor ring and hit ring
// with their heads and counts.
struct LeafState {
    uint32_t *ring, *cring;
    float4 *hits;
    uint32_t head, chead, hh;
    int nsq, ncq, nh;
};

// All 32 lanes: lane k tests both triangles of capsule survivor k (k < cnt)
// of the capsule ring, (u0, u1, u2) and (u3, u2, u1), its four texels loaded together;
// hits are compacted into the hit ring and weighed 32 at a time.
template <int TFMT, bool STATS, bool CLAMP>
__device__ __forceinline__ void test_quads(const MapDesc &d, const Query &q, LeafState &ls, int cnt, int lane,
                                           Acc &acc)
{
    const unsigned lt = (1u << lane) - 1u;
    bool h0 = false, h1 = false;
    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
    if (lane < cnt) {
        uint32_t pk = ls.cring[(ls.chead + uint32_t(lane)) & (kCapRing - 1)];
        int gi = int(pk >> 16), gj = int(pk & 0xffffu);
        float2 n0 = texel<TFMT>(d, gi, gj), n1 = texel<TFMT>(d, gi + 1, gj);
        float2 n2 = texel<TFMT>(d, gi, gj + 1), n3 = texel<TFMT>(d, gi + 1, gj + 1);
        uint32_t id = 2u * (uint32_t(gj) * uint32_t(d.n - 1) + uint32_t(gi));
        uint32_t hp = (uint32_t(gi) << 15) | (uint32_t(gj) << 1);
        float cr, e1, e2;
        h0 = edge_test<STATS, CLAMP>(q, n0, n1, n2, gi, gj, 1.f, id, acc, cr, e1, e2);
        if (h0) v0 = make_float4(cr, e1, e2, __uint_as_float(hp));
        h1 = edge_test<STATS, CLAMP>(q, n3, n2, n1, gi + 1, gj + 1, -1.f, id + 1u, acc, cr, e1, e2);
        if (h1) v1 = make_float4(cr, e1, e2, __uint_as_float(hp | 1u));
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {  // at most 31 + 32 entries queue between drains
        bool h = t ? h1 : h0;
        unsigned m = __ballot_sync(kFull, h);
        if (h) ls.hits[(ls.hh + uint32_t(ls.nh) + __popc(m & lt)) & (kHitRing - 1)] = t ? v1 : v0;
        ls.nh += __popc(m);
        __syncwarp();
        if (ls.nh >= 32) {
            drain_hits<STATS>(q, d.n, d.L, ls.hits, ls.hh, 32, lane, acc);
            ls.hh += 32;
            ls.nh -= 32;
            __syncwarp();
        }
    }
}

// Cluster triangle test (Sec. 4.2) in vertex-relative form: p = m - A,
// b = B - A, c = C - A.  Same rule as edge_test (closed bounding box, edge
// functions sign-consistent with the orientation); the Jacobian of the
// cluster map is cross / 4^l, applied when the hit is weighed.  Triangles
// with FP32 |cross| < 2e-10 are decided and weighed here in FP64.
template <bool STATS>
__device__ __forceinline__ bool cluster_edge_test(const Query &q, float2 p, float2 b, float2 c, int l, int ai,
                                                  int aj, float dir, uint32_t id, Acc &acc, float &cr_o, float &e1_o,
                                                  float &e2_o)
{
    if (STATS) acc.tests++;
    if (p.x < fminf(0.f, fminf(b.x, c.x)) || p.x > fmaxf(0.f, fmaxf(b.x, c.x)) ||
        p.y < fminf(0.f, fminf(b.y, c.y)) || p.y > fmaxf(0.f, fmaxf(b.y, c.y)))
        return false;
    float cr = dop(b.x, c.y, b.y, c.x);
    if (fabsf(cr) >= kTinyCross) {
        float e0 = dop(c.x - b.x, p.y - b.y, c.y - b.y, p.x - b.x);
        float e1 = dop(p.x, c.y, p.y, c.x);
        float e2 = dop(b.x, p.y, b.y, p.x);
        bool hit = cr > 0.f ? (e0 >= 0.f && e1 >= 0.f && e2 >= 0.f) : (e0 <= 0.f && e1 <= 0.f && e2 <= 0.f);
        cr_o = cr;
        e1_o = e1;
        e2_o = e2;
        return hit;
    }
    double bx = b.x, by = b.y, cx = c.x, cy = c.y, px = p.x, py = p.y;
    double dcr = bx * cy - by * cx;
    if (dcr == 0.0) {
        if (STATS) acc.degen++;
        return false;
    }
    if (STATS) acc.fp64++;
    acc.flags |= PNDF_QF_FP64;
    double e0 = (cx - bx) * (py - by) - (cy - by) * (px - bx);
    double e1 = px * cy - py * cx;
    double e2 = bx * py - by * px;
    bool hit = dcr > 0.0 ? (e0 >= 0.0 && e1 >= 0.0 && e2 >= 0.0) : (e0 <= 0.0 && e1 <= 0.0 && e2 <= 0.0);
    if (!hit) return false;
    double dl1 = e1 / dcr, dl2 = e2 / dcr;
    double dx = (double(ai) - double(q.x)) + dir * dl1;
    double dy = (double(aj) - double(q.y)) + dir * dl2;
    double qq = double(q.ia) * dx * dx + 2.0 * double(q.ib) * dx * dy + double(q.ic) * dy * dy;
    const double w = kweight_d(q, dx, qq);
    if (w == 0.0) return false;
    double sc = double(1u << l);
    acc_add(acc, float(w * sc * sc / fabs(dcr)));
    if (STATS) {
        acc.hits++;
        acc.hash += fmix32(id);
    }
    return false;
}

// All 32 lanes: lane k < cnt tests the two cluster triangles of the cut node
// in last[-k] (level, Morton): lower (c00, c10, c01) at uv (O, O + (a, 0),
// O + (0, a)), upper (c11, c01, c10) at (O + (a, a), O + (0, a), O + (a, 0)),
// a = 2^l; hits join the hit ring.
template <bool STATS>
__device__ __forceinline__ void test_clusters(const MapDesc &d, const ClusterDesc &cd, const Query &q,
                                              const uint32_t *last, int cnt, LeafState &ls, int lane, Acc &acc)
{
    const unsigned lt = (1u << lane) - 1u;
    bool h0 = false, h1 = false;
    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
    if (lane < cnt) {
        uint32_t ent = last[-lane];
        int l = int(ent >> 28);
        uint32_t m = ent & kMortonMask;
        const float4 *rec = cd.cl[l] + 2 * size_t(m);
        float4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
        int ox = int(compact1by1(m)) << l, oy = int(compact1by1(m >> 1)) << l;
        int a = 1 << l;
        float2 p = make_float2(q.mx - r0.x, q.my - r0.y);
        float2 d10 = make_float2(r0.z, r0.w), d01 = make_float2(r1.x, r1.y), d11 = make_float2(r1.z, r1.w);
        uint32_t tag = kClusterTag | (uint32_t(l) << 27) | (m << 1);
        // hit fingerprint id (stats): row-major node index at its level
        uint32_t id = kClusterTag | (uint32_t(l) << 27) |
                      (((uint32_t(oy >> l) << (d.L - l)) + uint32_t(ox >> l)) << 1);
        float cr, e1, e2;
        if (STATS) acc.clusters++;
        h0 = cluster_edge_test<STATS>(q, p, d10, d01, l, ox, oy, float(a), id, acc, cr, e1, e2);
        if (h0) v0 = make_float4(cr, e1, e2, __uint_as_float(tag));
        float2 pu = make_float2(p.x - d11.x, p.y - d11.y);
        float2 bu = make_float2(d01.x - d11.x, d01.y - d11.y), cu = make_float2(d10.x - d11.x, d10.y - d11.y);
        h1 = cluster_edge_test<STATS>(q, pu, bu, cu, l, ox + a, oy + a, -float(a), id | 1u, acc, cr, e1, e2);
        if (h1) v1 = make_float4(cr, e1, e2, __uint_as_float(tag | 1u));
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        bool h = t ? h1 : h0;
        unsigned mk = __ballot_sync(kFull, h);
        if (h) ls.hits[(ls.hh + uint32_t(ls.nh) + __popc(mk & lt)) & (kHitRing - 1)] = t ? v1 : v0;
        ls.nh += __popc(mk);
        __syncwarp();
        if (ls.nh >= 32) {
            drain_hits<STATS>(q, d.n, d.L, ls.hits, ls.hh, 32, lane, acc);
            ls.hh += 32;
            ls.nh -= 32;
            __syncwarp();
        }
    }
}

// Four level-0 boxes (Morton-consecutive quads) in one 32-byte (FP16) or
// 64-byte (FP32) load; returns bit u set when box u holds m.
template <int BFMT, bool CLAMP>
__device__ __forceinline__ unsigned quad_boxes_hold(const MapDesc &d, uint32_t first, const Query &q)
{
    const float mx = q.mx, my = q.my, rho = CLAMP ? q.rho : 0.f;
    unsigned bits = 0;
    if (BFMT == PNDF_BOUNDS_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(d.lv[0]) + first;
        float4 b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = __ldg(p + u);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            bits |= CLAMP ? unsigned(mx >= b[u].x - rho && mx <= b[u].z + rho && my >= b[u].y - rho &&
                                     my <= b[u].w + rho) << u
                          : unsigned(mx >= b[u].x && mx <= b[u].z && my >= b[u].y && my <= b[u].w) << u;
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint2 *>(d.lv[0]) + first);
        uint4 v0 = __ldg(p), v1 = __ldg(p + 1);
        uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 lo = __half22float2(*reinterpret_cast<__half2 *>(&w[2 * u]));
            float2 hi = __half22float2(*reinterpret_cast<__half2 *>(&w[2 * u + 1]));
            bits |= CLAMP ? unsigned(mx >= lo.x - rho && mx <= hi.x + rho && my >= lo.y - rho && my <= hi.y + rho) << u
                          : unsigned(mx >= lo.x && mx <= hi.x && my >= lo.y && my <= hi.y) << u;
        }
    }
    return bits;
}

// A stored node box decoded to (s_min, t_min, s_max, t_max).
template <int BFMT>
__device__ __forceinline__ float4 box_floats(const uint4 &v)
{
    if (BFMT == PNDF_BOUNDS_F32)
        return make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w));
    float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// All 32 lanes: lane k takes box survivors k and k + 32 of the ring (those
// below cnt <= 64; both quads' boxes and capsule codes are loaded before
// either is used), tests m against each quad's capsule, and the survivors
// are compacted into the capsule ring, whose quads are tested 32 at a time.
template <int BFMT, int TFMT, bool STATS, bool CLAMP>
__device__ __forceinline__ void capsule_round(const MapDesc &d, const Query &q, LeafState &ls, int cnt, int lane,
                                              Acc &acc)
{
    const unsigned lt = (1u << lane) - 1u;
    bool pass[2] = {false, false};
    uint32_t pk[2] = {0u, 0u};
    uint4 bx[2];
    uint2 code[2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
        if (lane + 32 * r < cnt) {
            pk[r] = ls.ring[(ls.head + uint32_t(lane + 32 * r)) & (kRing - 1)];
            const uint32_t mq = morton2(pk[r] >> 16, pk[r] & 0xffffu);
            bx[r] = node_box<BFMT>(d, 0, mq);
            code[r] = __ldg(d.qcap + mq);
        }
#pragma unroll
    for (int r = 0; r < 2; ++r)
        if (lane + 32 * r < cnt) {
            const float4 b = box_floats<BFMT>(bx[r]);
            const Capsule c = decode_capsule(b.x, b.y, b.z, b.w, code[r]);
            pass[r] = capsule_holds(c, q.mx, q.my, CLAMP ? c.w + q.rho : c.w);
        }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const unsigned m = __ballot_sync(kFull, pass[r]);
        if (pass[r]) ls.cring[(ls.chead + uint32_t(ls.ncq) + __popc(m & lt)) & (kCapRing - 1)] = pk[r];
        ls.ncq += __popc(m);
        __syncwarp();
        if (ls.ncq >= 32) {
            test_quads<TFMT, STATS, CLAMP>(d, q, ls, 32, lane, acc);
            ls.chead += 32;
            ls.ncq -= 32;
            __syncwarp();
        }
    }
}

// All 32 lanes: filter the queued leaf blocks' quads by their level-0 boxes
// (lane t: quads 4 (t & 3) .. 4 (t & 3) + 3 of block p + (t >> 2), eight
// blocks per pass), compact the survivors into the ring with ballot/popc and
// test them 32 quads (64 triangles) at a time.
template <int BFMT, int TFMT, bool STATS, bool CLAMP>
__device__ __forceinline__ void process_leaves(const MapDesc &d, const Query &q, const uint32_t *lq, int nleaf,
                                               LeafState &ls, int lane, Acc &acc)
{
    const unsigned lt = (1u << lane) - 1u;
    for (int p = 0; p < nleaf; p += 8) {
        const int blk = p + (lane >> 2);
        unsigned bits = 0;
        uint32_t base = 0;
        if (blk < nleaf) {
            uint32_t m = lq[blk] & kMortonMask;
            // the lane's four quads are the 2 x 2 quad group (lane & 3) of the
            // block (Morton order): (i0 + u & 1, j0 + u >> 1) for u = 0..3
            const uint32_t i0 = compact1by1(m) * kLeafQuads + ((uint32_t(lane) & 1u) << 1);
            const uint32_t j0 = compact1by1(m >> 1) * kLeafQuads + (uint32_t(lane) & 2u);
            base = (i0 << 16) | j0;
            bits = quad_boxes_hold<BFMT, CLAMP>(d, (m << 4) | (uint32_t(lane & 3) << 2), q);
            if (STATS) {
                acc.quads += 4;
                if ((lane & 3) == 0) acc.leaves++;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            bool pass = (bits >> u) & 1u;
            unsigned m = __ballot_sync(kFull, pass);
            if (pass)
                ls.ring[(ls.head + uint32_t(ls.nsq) + __popc(m & lt)) & (kRing - 1)] =
                    base + ((uint32_t(u) & 1u) << 16) + (uint32_t(u) >> 1);
            ls.nsq += __popc(m);
        }
        __syncwarp();
        while (ls.nsq >= 64) {
            capsule_round<BFMT, TFMT, STATS, CLAMP>(d, q, ls, 64, lane, acc);
            ls.head += 64;
            ls.nsq -= 64;
            __syncwarp();
        }
    }
}

// Nodes of size sz (S per side) whose closed extent [a sz, (a+1) sz] meets
// [x - r, x + r]; clamped in float first so no int conversion can overflow.
// Empty (a0 > a1) when the interval misses the map.
__device__ __forceinline__ void node_range(float x, float r, float sz, int S, int &a0, int &a1)
{
    float f0 = fmaxf(ceilf((x - r) / sz) - 1.0f, 0.0f);
    float f1 = fminf(floorf((x + r) / sz), float(S - 1));
    if (!(f0 <= f1)) {
        a0 = 1;
        a1 = 0;
        return;
    }
    a0 = int(f0);
    a1 = int(f1);
}

__device__ __forceinline__ int entry_level(const Query &q, int L)
{
    float r = fmaxf(q.rx, q.ry);
    int l = kLeafLevel;
    while (l < L && float(1u << l) < r) ++l;
    return l;
}

// The hierarchical descent from the nodes [a0, a1] x [c0, c1] of level e
// (at most 4 x 4 of them) into the lane's accumulator: the whole query when
// they are its entry nodes, one tile of it when a large footprint is divided
// among warps.  Node boxes nest (a parent's normal box and uv box contain its
// children's), so a leaf block is reached from any level above it exactly
// when every node test on its path passes: the hit set, and with the exact
// sum the result, does not depend on the level the descent starts from.
template <int BFMT, int TFMT, bool STATS, bool CLUSTER, bool CLAMP>
__device__ __forceinline__ void eval_range(const MapDesc &d, const ClusterDesc &cd, const Query &q, int e, int a0,
                                           int a1, int c0, int c1, int lane, uint32_t *stk, uint32_t *lq,
                                           uint32_t *ring, float4 *hits, Acc &acc)
{
    int top = 0, nleaf = 0, ncl = 0;
    const unsigned lt = (1u << lane) - 1u;
    // entry nodes: at most 4 x 4
    {
        int a = a0 + (lane & 3), c = c0 + (lane >> 2);
        bool valid = lane < 16 && a <= a1 && c <= c1;
        bool pass = valid && node_test<BFMT, CLAMP>(d, q, e, a, c);
        bool inside = pass && node_inside(q, e, a, c);
        bool cut = false;
        if (STATS) acc.nodes += valid ? 1u : 0u;
        if (CLUSTER && pass) {  // the cut of Sec. 4.2: e <= r_x r_y tau
            cut = __ldg(cd.ce[e] + morton2(a, c)) <= q.theta;
            if (STATS) acc.cchecks++;
        }
        unsigned m = __ballot_sync(kFull, pass && !cut);
        unsigned mc = __ballot_sync(kFull, cut);
        if (pass && !cut) {
            int pos = __popc(m & lt);
            uint32_t ent = pack(e, inside, morton2(a, c));
            if (e == kLeafLevel)
                lq[pos] = ent;
            else
                stk[pos] = ent;
        }
        if (CLUSTER && cut) lq[kLeafQ - 1 - __popc(mc & lt)] = pack(e, false, morton2(a, c));
        if (e == kLeafLevel)
            nleaf = __popc(m);
        else
            top = __popc(m);
        ncl = __popc(mc);
        __syncwarp();
    }
    bool overflow = false;
    LeafState ls{ring, ring + kRing, hits, 0u, 0u, 0u, 0, 0, 0};
    while (true) {
        // leaf blocks are filtered eight to a pass (four lanes each): while
        // the stack still holds nodes only whole passes run, and the rest
        // (fewer than 8) waits at the front of the queue for the next step
        const int nrun = top == 0 ? nleaf : (nleaf & ~7);
        process_leaves<BFMT, TFMT, STATS, CLAMP>(d, q, lq, nrun, ls, lane, acc);
        if (nrun > 0 && nrun < nleaf) {
            const int rest = nleaf - nrun;  // < 8 <= nrun: source and target do not overlap
            uint32_t v = lane < rest ? lq[nrun + lane] : 0u;
            if (lane < rest) lq[lane] = v;
            __syncwarp();
        }
        nleaf -= nrun;
        if (CLUSTER) {
            // cut nodes sit at the back of the leaf queue
            for (int k0 = 0; k0 < ncl; k0 += 32) {
                test_clusters<STATS>(d, cd, q, lq + kLeafQ - 1 - k0, min(32, ncl - k0), ls, lane, acc);
                __syncwarp();
            }
            ncl = 0;
        }
        if (top == 0) break;
        // pop up to 16 nodes; lane k tests child (k & 3) of popped nodes
        // (k >> 2) and (k >> 2) + 8, so two box loads per lane are in flight
        int npop = min(top, 16);
        top -= npop;
        bool pass[2], ins[2], cut[2] = {false, false};
        int cl[2];
        uint32_t cm[2];
        uint4 bx[2];
        float ev[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int slot = (lane >> 2) + 8 * r;
            uint32_t ent = slot < npop ? stk[top + slot] : 0u;
            cl[r] = int(ent >> 28) - 1;
            cm[r] = ((ent & kMortonMask) << 2) | uint32_t(lane & 3);
            ins[r] = (ent >> 27) & 1u;
            pass[r] = slot < npop;
            if (STATS && slot < npop) acc.nodes++;
        }
        // both box loads issue before the uv tests, which hide their latency
        // (895.9 ms against 915.2 ms per 4M-query flake step, same bits)
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (pass[r]) {
                bx[r] = node_box<BFMT>(d, cl[r], cm[r]);
                if (CLUSTER) ev[r] = __ldg(cd.ce[cl[r]] + cm[r]);
            }
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (pass[r] && !ins[r]) {
                // parent straddles the ellipse: test this child's uv box
                uint32_t a = compact1by1(cm[r]), c = compact1by1(cm[r] >> 1);
                pass[r] = node_in_footprint(q, cl[r], a, c);
                ins[r] = pass[r] && node_inside(q, cl[r], a, c);
            }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            pass[r] = pass[r] && stored_box_holds<BFMT, CLAMP>(bx[r], q);
            if (CLUSTER && pass[r]) {  // the cut of Sec. 4.2: e <= r_x r_y tau
                cut[r] = ev[r] <= q.theta;
                if (STATS) acc.cchecks++;
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            bool to_leaf = pass[r] && !cut[r] && cl[r] == kLeafLevel;
            bool to_stack = pass[r] && !cut[r] && cl[r] > kLeafLevel;
            unsigned ml = __ballot_sync(kFull, to_leaf);
            unsigned ms = __ballot_sync(kFull, to_stack);
            if (CLUSTER) {
                unsigned mc = __ballot_sync(kFull, cut[r]);
                if (cut[r]) lq[kLeafQ - 1 - ncl - __popc(mc & lt)] = pack(cl[r], false, cm[r]);
                ncl += __popc(mc);
            }
            if (to_leaf) lq[nleaf + __popc(ml & lt)] = pack(cl[r], ins[r], cm[r]);
            if (to_stack) {
                int pos = top + __popc(ms & lt);
                if (pos < kStackCap) stk[pos] = pack(cl[r], ins[r], cm[r]);
            }
            nleaf += __popc(ml);
            top += __popc(ms);
            if (top > kStackCap) {
                top = kStackCap;
                overflow = true;
            }
        }
        __syncwarp();
    }
    if (ls.nsq > 0) capsule_round<BFMT, TFMT, STATS, CLAMP>(d, q, ls, ls.nsq, lane, acc);  // nsq < 64 here
    if (ls.ncq > 0) test_quads<TFMT, STATS, CLAMP>(d, q, ls, ls.ncq, lane, acc);  // ncq < 32 here
    if (ls.nh > 0) drain_hits<STATS>(q, d.n, d.L, ls.hits, ls.hh, ls.nh, lane, acc);  // nh < 32 here
    if (overflow) acc.flags |= PNDF_QF_OVERFLOW;
}

// Warp total of the lanes' accumulators: the fixed-point sum (exact), the
// flags and, with STATS, the counters (all lanes hold the result).
template <bool STATS>
__device__ __forceinline__ void warp_total(Acc &acc, unsigned long long &lo, unsigned long long &hi, uint32_t &fl)
{
    lo = s_sum_lo[threadIdx.x];
    hi = s_sum_hi[threadIdx.x];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long lo_o = __shfl_xor_sync(kFull, lo, off);
        const unsigned long long hi_o = __shfl_xor_sync(kFull, hi, off);
        lo += lo_o;
        const unsigned long long h0 = hi;
        hi += hi_o + (lo < lo_o ? 1ull : 0ull);
        if (hi < h0) acc.flags |= kHuge;
    }
    fl = __reduce_or_sync(kFull, acc.flags);
    if (STATS) {
        acc.hits = __reduce_add_sync(kFull, acc.hits);
        acc.hash = __reduce_add_sync(kFull, acc.hash);
        acc.tests = __reduce_add_sync(kFull, acc.tests);
        acc.fp64 = __reduce_add_sync(kFull, acc.fp64);
        acc.degen = __reduce_add_sync(kFull, acc.degen);
        acc.nodes = __reduce_add_sync(kFull, acc.nodes);
        acc.leaves = __reduce_add_sync(kFull, acc.leaves);
        acc.quads = __reduce_add_sync(kFull, acc.quads);
        acc.cchecks = __reduce_add_sync(kFull, acc.cchecks);
        acc.clusters = __reduce_add_sync(kFull, acc.clusters);
    }
}

// KERN: the footprint kernel (pndf_kernel), a compile-time constant so the
// query's kernel fields and branches fold away (each kernel is its own
// instantiation).
template <int BFMT, int TFMT, bool STATS, bool FLAT, bool CLUSTER, int KERN>
__device__ void eval_one(const MapDesc &d, const ClusterDesc &cd, float tau, float jac_eps, const pndf_query &rec,
                         int lane, uint32_t *stk, uint32_t *lq, uint32_t *ring, float4 *hits, float &D_out,
                         uint32_t &flags_out, pndf_query_stats *st_out)
{
    constexpr bool CLAMP = KERN == kKernGaussClamp;
    Query q = make_query(rec, KERN, jac_eps);
    Acc acc = {};
    acc_zero();
    if (!q.valid) {
        if (lane == 0) {
            D_out = __int_as_float(0x7fc00000);
            flags_out = PNDF_QF_INVALID;
            record_status(d.status, &g_status_eval, PNDF_QF_INVALID);
            if (STATS) *st_out = pndf_query_stats{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        }
        return;
    }
    if (CLUSTER) q.theta *= tau;  // r_x r_y tau with the support's half-widths
    const int L = d.L;
    if (FLAT) {
        // every leaf block meeting the 4-sigma box, no pruning
        const int S = 1 << (L - kLeafLevel);
        const float sz = float(kLeafQuads);
        int a0, a1, c0, c1;
        node_range(q.x, q.rx, sz, S, a0, a1);
        node_range(q.y, q.ry, sz, S, c0, c1);
        for (int c = c0; c <= c1; ++c)
            for (int a = a0; a <= a1; ++a)
                test_leaf<STATS>(d, q, a, c, leaf_texel<TFMT>(d, a, c, lane), lane, acc);
    } else {
        const int e = entry_level(q, L);
        const int S = 1 << (L - e);
        const float sz = float(1u << e);
        int a0, a1, c0, c1;
        node_range(q.x, q.rx, sz, S, a0, a1);
        node_range(q.y, q.ry, sz, S, c0, c1);
        eval_range<BFMT, TFMT, STATS, CLUSTER, CLAMP>(d, cd, q, e, a0, a1, c0, c1, lane, stk, lq, ring, hits, acc);
    }
    unsigned long long lo, hi;
    uint32_t fl;
    warp_total<STATS>(acc, lo, hi, fl);
    if (lane == 0) {
        D_out = acc_value(lo, hi, fl);
        fl &= ~kHuge;
        flags_out = fl;
        if (fl & PNDF_QF_OVERFLOW) record_status(d.status, &g_status_eval, PNDF_QF_OVERFLOW);
        if (STATS)
            *st_out = pndf_query_stats{acc.nodes, acc.leaves, acc.tests, acc.hits,    acc.hash,
                                       acc.fp64,  acc.degen,  acc.quads, acc.cchecks, acc.clusters};
    }
}

__constant__ ClusterDesc kNoClusters;  // never read: the variants without the cut

// ---- large footprints divided among warps ----
//
// One warp per query leaves a batch waiting on its largest footprints: a
// sigma = 1024 query on a 16384^2 map is about 100 ms of one warp, longer
// than the rest of a few-thousand-query batch together.  Before the
// traversal, split_work sums a work estimate over the batch (the area of each
// support's bounding box) and split_plan divides every query whose estimate
// is more than twice the target w_t = max(W / (4 x resident warps), 2.6e5)
// (2.6e5: the box of a sigma = 64 footprint) into tiles of at most 4 x 4
// nodes of one level, the deepest level (>= 4, at most 256 tiles) whose tile
// count reaches its estimate / w_t.  The traversal hands out the tiles first
// (largest queries first), then the undivided queries; the last warp to
// finish a query's tiles writes its result.  The sum is exact, so the
// result is the same bits whichever way the query was divided.
constexpr int kSplitMinLevel = 4;
constexpr uint32_t kSplitMaxTiles = 256;
constexpr float kSplitMinWork = 2.6e5f;
constexpr int kSplitPerWarp = 4;

struct SplitEntry {
    uint32_t qi, tiles;        // the query (caller index) and its tile count
    unsigned long long base;   // index of its first tile among all tiles
    int32_t level, pad;        // node level of the tiles
    unsigned long long lo, hi; // fixed-point sum of the finished tiles
    uint32_t done, flags;      // tiles finished; OR of their flags
    pndf_query_stats st;       // summed counters (stats launches)
};

struct SplitPlan {
    SplitEntry *entries;       // null: no division
    uint8_t *marker;           // per query (caller index): 1 = divided into tiles
    unsigned long long *ctr;   // (entries << 40) | tiles reserved
    double *work;              // the batch's summed estimate
    float *wt;                 // the target w_t (served steps: written by the plan for the step kernel)
    uint32_t cap;              // entries capacity
    int resident_warps;
};

__device__ __forceinline__ float split_estimate(const Query &q)
{
    return q.valid ? 64.f + 4.f * q.rx * q.ry : 64.f;
}

template <int KERN>
__global__ void split_work(const pndf_query *__restrict__ qs, int64_t nq, float jac_eps, double *__restrict__ work)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nq; k += int64_t(gridDim.x) * blockDim.x)
        acc += double(split_estimate(make_query(qs[k], KERN, jac_eps)));
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(work, red[0]);
}

// Tiles of level l over the support's bounding box: ceil(nx / 4) ceil(ny / 4).
__device__ __forceinline__ uint32_t split_tiles(const Query &q, int L, int l, int &a0, int &a1, int &c0, int &c1)
{
    const int S = 1 << (L - l);
    const float sz = float(1u << l);
    node_range(q.x, q.rx, sz, S, a0, a1);
    node_range(q.y, q.ry, sz, S, c0, c1);
    if (a0 > a1 || c0 > c1) return 0u;
    return uint32_t((a1 - a0) / 4 + 1) * uint32_t((c1 - c0) / 4 + 1);
}

__device__ __forceinline__ float split_target(const SplitPlan &p)
{
    return fmaxf(float(*p.work / (double(kSplitPerWarp) * p.resident_warps)), kSplitMinWork);
}

// Whether query q is divided at target wt, and into which tiles: the deepest
// level (>= kSplitMinLevel) whose tile count stays <= kSplitMaxTiles, or the
// first going down whose count reaches estimate / wt; at least two tiles.
__device__ __forceinline__ bool split_choice(const Query &q, int L, float wt, int &level, uint32_t &tiles)
{
    const float w = split_estimate(q);
    if (!q.valid || !(w > 2.f * wt)) return false;
    const float target = w / wt;
    int best = -1, a0, a1, c0, c1;
    uint32_t bt = 0;
    for (int l = entry_level(q, L) - 1; l >= kSplitMinLevel; --l) {
        const uint32_t t = split_tiles(q, L, l, a0, a1, c0, c1);
        if (t > kSplitMaxTiles) break;
        best = l;
        bt = t;
        if (float(t) >= target) break;
    }
    level = best;
    tiles = bt;
    return best >= 0 && bt >= 2;
}

// Reserve an entry and its tiles; false if the entries are full (never
// expected: the division bounds them by 2 x the resident warps).
__device__ __forceinline__ bool split_reserve(const SplitPlan &p, uint32_t qi, int seg, int level, uint32_t tiles)
{
    const unsigned long long old = atomicAdd(p.ctr, (1ull << 40) | tiles);
    const unsigned long long idx = old >> 40;
    if (idx >= p.cap) return false;
    SplitEntry &E = p.entries[idx];
    E.qi = qi;
    E.tiles = tiles;
    E.base = old & ((1ull << 40) - 1ull);
    E.level = level;
    E.pad = seg;
    E.lo = E.hi = 0ull;
    E.done = E.flags = 0u;
    E.st = pndf_query_stats{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    return true;
}

template <int KERN>
__global__ void split_plan(MapDesc d, const pndf_query *__restrict__ qs, int64_t nq, float jac_eps, SplitPlan p)
{
    const float wt = split_target(p);
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nq; k += int64_t(gridDim.x) * blockDim.x) {
        const Query q = make_query(qs[k], KERN, jac_eps);
        int level;
        uint32_t tiles;
        p.marker[k] = split_choice(q, d.L, wt, level, tiles) && split_reserve(p, uint32_t(k), 0, level, tiles);
    }
}

// Work index k < ntiles: the entry of the divided query it belongs to (the
// last entry whose first tile is <= k) and the tile's node range.
__device__ __forceinline__ int tile_entry(const SplitPlan &p, int n_entries, unsigned long long k)
{
    int lo = 0, hi = n_entries - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&p.entries[mid].base) <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void tile_range(const Query &q, int L, int l, uint32_t j, int &a0, int &a1, int &c0, int &c1)
{
    int b0, b1, d0, d1;
    split_tiles(q, L, l, b0, b1, d0, d1);
    const int ntx = (b1 - b0) / 4 + 1;
    a0 = b0 + 4 * int(j % uint32_t(ntx));
    c0 = d0 + 4 * int(j / uint32_t(ntx));
    a1 = min(b1, a0 + 3);
    c1 = min(d1, c0 + 3);
}

// Lane 0: fold a tile's warp total into its query's entry; the warp that
// folds in the last tile writes D, the flags and the counters.
template <bool STATS>
__device__ __forceinline__ void tile_finish(const MapDesc &d, SplitEntry &E, const Acc &acc, unsigned long long lo,
                                            unsigned long long hi, uint32_t fl, float *D, uint32_t *flags,
                                            pndf_query_stats *stats)
{
    const unsigned long long old = atomicAdd(&E.lo, lo);
    const unsigned long long add_hi = hi + (old + lo < old ? 1ull : 0ull);
    const unsigned long long old_hi = atomicAdd(&E.hi, add_hi);
    if (old_hi + add_hi < old_hi) fl |= kHuge;
    if (fl) atomicOr(&E.flags, fl);
    if (STATS) {
        atomicAdd(&E.st.nodes, acc.nodes);
        atomicAdd(&E.st.leaf_blocks, acc.leaves);
        atomicAdd(&E.st.tri_tests, acc.tests);
        atomicAdd(&E.st.hits, acc.hits);
        atomicAdd(&E.st.hit_hash, acc.hash);
        atomicAdd(&E.st.fp64_tris, acc.fp64);
        atomicAdd(&E.st.degenerate, acc.degen);
        atomicAdd(&E.st.quads, acc.quads);
    }
    __threadfence();
    if (atomicAdd(&E.done, 1u) == __ldg(&E.tiles) - 1u) {
        __threadfence();
        const uint32_t qi = __ldg(&E.qi);
        const uint32_t f = __ldcg(&E.flags);
        D[qi] = acc_value(__ldcg(&E.lo), __ldcg(&E.hi), f);
        if (flags) flags[qi] = f & ~kHuge;
        if (f & PNDF_QF_OVERFLOW) record_status(d.status, &g_status_eval, PNDF_QF_OVERFLOW);
        if (STATS)
            stats[qi] = pndf_query_stats{__ldcg(&E.st.nodes),      __ldcg(&E.st.leaf_blocks), __ldcg(&E.st.tri_tests),
                                         __ldcg(&E.st.hits),       __ldcg(&E.st.hit_hash),    __ldcg(&E.st.fp64_tris),
                                         __ldcg(&E.st.degenerate), __ldcg(&E.st.quads),       0u,
                                         0u};
    }
}

template <int BFMT, int TFMT, bool STATS, bool FLAT, bool CLUSTER, int KERN>
__global__ void __launch_bounds__(256, PNDF_TRAVERSE_MIN_CTAS)
    traverse_kernel(MapDesc d, ClusterDesc cd, float tau, float jac_eps, const pndf_query *__restrict__ qs,
                    const uint32_t *__restrict__ order, int64_t nq, float *__restrict__ D,
                    uint32_t *__restrict__ flags, pndf_query_stats *__restrict__ stats,
                    unsigned long long *__restrict__ cursor, SplitPlan sp)
{
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *stk = smem + warp * kWarpSmemWords;
    uint32_t *lq = stk + kStackCap;
    uint32_t *ring = lq + kLeafQ;
    float4 *hits = reinterpret_cast<float4 *>(ring + kRing + kCapRing);
    // the divided queries' tiles take the first s_ntiles work indices
    __shared__ unsigned long long s_ntiles;
    __shared__ int s_entries;
    __shared__ uint32_t s_dest[8][2];  // per warp: query, entry (-1: whole query)
    if (threadIdx.x == 0) {
        int n = 0;
        unsigned long long t = 0ull;
        if (!FLAT && !CLUSTER && sp.entries) {
            n = int(min(__ldcg(sp.ctr) >> 40, (unsigned long long)sp.cap));
            if (n > 0) t = __ldcg(&sp.entries[n - 1].base) + __ldcg(&sp.entries[n - 1].tiles);
        }
        s_entries = n;
        s_ntiles = t;
    }
    __syncthreads();
    while (true) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(cursor, 1ull);
        k = __shfl_sync(kFull, k, 0);
        if (FLAT || CLUSTER) {
            if (k >= (unsigned long long)nq) break;
            const int64_t qi = order ? int64_t(order[k]) : int64_t(k);
            float Dv;
            uint32_t fv;
            eval_one<BFMT, TFMT, STATS, FLAT, CLUSTER, KERN>(d, cd, tau, jac_eps, qs[qi], lane, stk, lq, ring, hits, Dv,
                                                             fv, stats ? stats + qi : nullptr);
            if (lane == 0) {
                D[qi] = Dv;
                if (flags) flags[qi] = fv;
            }
            continue;
        }
        // a tile of a divided query, or a whole query: one descent either way
        constexpr bool CLAMP = KERN == kKernGaussClamp;
        int ei = -1;  // the divided query's entry, or -1 for a whole query
        uint32_t qi;
        Query q;
        int e, a0, a1, c0, c1;
        if (k < s_ntiles) {
            ei = tile_entry(sp, s_entries, k);
            const SplitEntry &E = sp.entries[ei];
            qi = __ldg(&E.qi);
            q = make_query(qs[qi], KERN, jac_eps);
            e = __ldg(&E.level);
            tile_range(q, d.L, e, uint32_t(k - __ldg(&E.base)), a0, a1, c0, c1);
        } else {
            k -= s_ntiles;
            if (k >= (unsigned long long)nq) break;
            qi = order ? order[k] : uint32_t(k);
            if (s_entries > 0 && sp.marker[qi]) continue;  // evaluated as tiles
            q = make_query(qs[qi], KERN, jac_eps);
            if (!q.valid) {
                if (lane == 0) {
                    D[qi] = __int_as_float(0x7fc00000);
                    if (flags) flags[qi] = PNDF_QF_INVALID;
                    record_status(d.status, &g_status_eval, PNDF_QF_INVALID);
                    if (STATS) stats[qi] = pndf_query_stats{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
                }
                continue;
            }
            e = entry_level(q, d.L);
            const float sz = float(1u << e);
            node_range(q.x, q.rx, sz, 1 << (d.L - e), a0, a1);
            node_range(q.y, q.ry, sz, 1 << (d.L - e), c0, c1);
        }
        // where the result goes waits in shared memory during the descent
        if (lane == 0) {
            s_dest[warp][0] = qi;
            s_dest[warp][1] = uint32_t(ei);
        }
        Acc acc = {};
        acc_zero();
        eval_range<BFMT, TFMT, STATS, false, CLAMP>(d, cd, q, e, a0, a1, c0, c1, lane, stk, lq, ring, hits, acc);
        unsigned long long lo, hi;
        uint32_t fl;
        warp_total<STATS>(acc, lo, hi, fl);
        if (lane == 0) {
            qi = s_dest[warp][0];
            ei = int(s_dest[warp][1]);
            if (ei >= 0) {
                tile_finish<STATS>(d, sp.entries[ei], acc, lo, hi, fl, D, flags, stats);
            } else {
                D[qi] = acc_value(lo, hi, fl);
                if (flags) flags[qi] = fl & ~kHuge;
                if (fl & PNDF_QF_OVERFLOW) record_status(d.status, &g_status_eval, PNDF_QF_OVERFLOW);
                if (STATS)
                    stats[qi] = pndf_query_stats{acc.nodes, acc.leaves, acc.tests, acc.hits,    acc.hash,
                                                 acc.fp64,  acc.degen,  acc.quads, acc.cchecks, acc.clusters};
            }
        }
    }
}

// ---- query keying and counting sort ----

// Sort key: entry level (largest footprints first, 4 bits), then a sub-key of
// `sub` bits (6..14, more for larger batches): the footprint centre's tile
// (mode 1), the query normal's bin over [-0.4, 0.4]^2 (mode 2), or both, tile
// major (mode 3) or normal-bin major (mode 4).  Grouping queries that share a
// region and a normal makes the warps in flight visit the same nodes and leaf
// blocks, so they share L1/L2 lines.  The order never changes a result.
__device__ __forceinline__ uint32_t sort_key(const MapDesc &d, const pndf_query &r, int mode, int sub)
{
    Query q = make_query(r);
    if (!q.valid) return 0u;
    int e = entry_level(q, d.L);
    int tb, mb;  // bits per axis for the tile and the normal bin
    if (mode == 1) {
        tb = sub >> 1;
        mb = 0;
    } else if (mode == 2) {
        tb = 0;
        mb = sub >> 1;
    } else {
        tb = (sub + 2) >> 2;
        mb = (sub >> 1) - tb;
    }
    float ts = float(1 << tb) / float(d.n), ms = float(1 << mb) / 0.8f;
    uint32_t tx = uint32_t(fminf(fmaxf(r.x * ts, 0.f), float((1 << tb) - 1)));
    uint32_t ty = uint32_t(fminf(fmaxf(r.y * ts, 0.f), float((1 << tb) - 1)));
    uint32_t mx = uint32_t(fminf(fmaxf((r.ms + 0.4f) * ms, 0.f), float((1 << mb) - 1)));
    uint32_t my = uint32_t(fminf(fmaxf((r.mt + 0.4f) * ms, 0.f), float((1 << mb) - 1)));
    uint32_t t = morton2(tx, ty), m = morton2(mx, my);
    uint32_t k = mode == 4 ? (m << (2 * tb)) | t : (t << (2 * mb)) | m;
    return (uint32_t(15 - e) << sub) | k;
}

// Sub-key bits for a batch of nq queries: about 16 queries per bin on average.
inline int sort_sub_bits(int64_t nq)
{
    int b = 6;
    while (b < kMaxSubBits && (int64_t(1) << (b + 4 + 2)) * 16 <= nq) b += 2;
    return b;
}

__global__ void key_hist(MapDesc d, const pndf_query *__restrict__ qs, int64_t nq, int mode, int sub,
                         uint32_t *__restrict__ keys, uint32_t *__restrict__ hist)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nq; k += int64_t(gridDim.x) * blockDim.x) {
        uint32_t key = sort_key(d, qs[k], mode, sub);
        keys[k] = key;
        atomicAdd(&hist[key], 1u);
    }
}

// One CTA of 1024 threads: exclusive scan of nbins (a multiple of 4096) counts
// in place, 4096 bins per round, four consecutive bins per thread.
__global__ void __launch_bounds__(1024) key_scan(uint32_t *__restrict__ hist, int nbins)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nbins; base += 4096) {
        uint4 v = reinterpret_cast<uint4 *>(hist + base)[threadIdx.x];
        uint32_t sum = v.x + v.y + v.z + v.w;
        uint32_t incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_tot[lane], wi = w;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                uint32_t t = __shfl_up_sync(kFull, wi, off);
                if (lane >= off) wi += t;
            }
            warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
        }
        __syncthreads();
        uint32_t run = carry_s + warp_tot[warp] + incl - sum;
        uint4 o;
        o.x = run;
        o.y = o.x + v.x;
        o.z = o.y + v.y;
        o.w = o.z + v.z;
        reinterpret_cast<uint4 *>(hist + base)[threadIdx.x] = o;
        __syncthreads();
        if (threadIdx.x == 1023) carry_s = run + sum;
        __syncthreads();
    }
}

__global__ void key_place(const uint32_t *__restrict__ keys, int64_t nq, uint32_t *__restrict__ offsets,
                          uint32_t *__restrict__ order)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nq; k += int64_t(gridDim.x) * blockDim.x) {
        uint32_t pos = atomicAdd(&offsets[keys[k]], 1u);
        order[pos] = uint32_t(k);
    }
}

// Key, histogram, scan and placement: order receives a permutation of 0..nq-1.
// scratch: hist (zeroed by the caller, 1 << (4 + sub) bins) and keys (nq).
cudaError_t sort_launch(const MapDesc &d, const pndf_query *q, int64_t nq, int mode, uint32_t *hist, uint32_t *keys,
                        uint32_t *order, cudaStream_t s)
{
    const int sub = sort_sub_bits(nq);
    int nbins = 1 << (4 + sub);
    if (nbins < 4096) nbins = 4096;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (nq + 255) / 256;
    if (blocks > int64_t(sms) * 8) blocks = int64_t(sms) * 8;
    key_hist<<<unsigned(blocks), 256, 0, s>>>(d, q, nq, mode, sub, keys, hist);
    key_scan<<<1, 1024, 0, s>>>(hist, nbins);
    key_place<<<unsigned(blocks), 256, 0, s>>>(keys, nq, hist, order);
    count_launches(3);
    return cudaGetLastError();
}

// Histogram bytes a batch of nq queries needs (a multiple of 16 KiB).
inline size_t sort_hist_bytes(int64_t nq)
{
    size_t bins = size_t(1) << (4 + sort_sub_bits(nq));
    if (bins < 4096) bins = 4096;
    return bins * sizeof(uint32_t);
}

template <int BFMT, int TFMT, bool STATS, bool FLAT, bool CLUSTER, int KERN>
cudaError_t launch_traverse(const MapDesc &d, const ClusterDesc &cd, float tau, float jac_eps, const pndf_query *q,
                            const uint32_t *order, int64_t nq, float *D, uint32_t *flags, pndf_query_stats *stats,
                            unsigned long long *cursor, int warps, int ctas_per_sm, SplitPlan sp, cudaStream_t s)
{
    if (FLAT || CLUSTER) sp.entries = nullptr;  // whole queries only (the cut depends on the entry level)
    auto kern = traverse_kernel<BFMT, TFMT, STATS, FLAT, CLUSTER, KERN>;
    int threads = warps * 32;
    size_t smem = size_t(warps) * kWarpSmemWords * sizeof(uint32_t);
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // with its static arrays the kernel passes the 48 KB a launch gets by default
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
    int64_t want = (nq + warps - 1) / warps;
    int64_t grid = int64_t(sms) * occ;
    if (sp.entries) {
        // the plan: the batch's work, then the division of its large footprints
        sp.resident_warps = int(grid) * warps;
        int64_t blocks = (nq + 255) / 256;
        if (blocks > int64_t(sms) * 8) blocks = int64_t(sms) * 8;
        split_work<KERN><<<unsigned(blocks), 256, 0, s>>>(q, nq, jac_eps, sp.work);
        split_plan<KERN><<<unsigned(blocks), 256, 0, s>>>(d, q, nq, jac_eps, sp);
        count_launches(2);
    } else if (grid > want) {
        grid = want;
    }
    if (grid < 1) grid = 1;
    kern<<<unsigned(grid), threads, smem, s>>>(d, cd, tau, jac_eps, q, order, nq, D, flags, stats, cursor, sp);
    count_launches(1);
    return cudaGetLastError();
}

template <int BFMT, int TFMT, int KERN>
cudaError_t dispatch_kernel(const MapDesc &d, const ClusterDesc &cd, const pndf_query *q, const uint32_t *order,
                            int64_t nq, float *D, uint32_t *flags, pndf_query_stats *stats,
                            unsigned long long *cursor, const pndf_eval_config &cfg, const SplitPlan &sp,
                            cudaStream_t s)
{
    const int warps = cfg.warps_per_cta > 0 ? cfg.warps_per_cta : 8;
    const int cps = cfg.ctas_per_sm;
    const float tau = cfg.tau;
    if (cfg.mode == PNDF_MODE_FLAT)
        return stats ? launch_traverse<BFMT, TFMT, true, true, false, KERN>(d, cd, 0.f, cfg.jac_eps, q, order, nq, D, flags, stats,
                                                                             cursor, warps, cps, sp, s)
                     : launch_traverse<BFMT, TFMT, false, true, false, KERN>(d, cd, 0.f, cfg.jac_eps, q, order, nq, D, flags, stats,
                                                                              cursor, warps, cps, sp, s);
    if (tau > 0.f)
        return stats ? launch_traverse<BFMT, TFMT, true, false, true, KERN>(d, cd, tau, cfg.jac_eps, q, order, nq, D, flags, stats,
                                                                             cursor, warps, cps, sp, s)
                     : launch_traverse<BFMT, TFMT, false, false, true, KERN>(d, cd, tau, cfg.jac_eps, q, order, nq, D, flags, stats,
                                                                              cursor, warps, cps, sp, s);
    return stats ? launch_traverse<BFMT, TFMT, true, false, false, KERN>(d, cd, 0.f, cfg.jac_eps, q, order, nq, D, flags, stats,
                                                                          cursor, warps, cps, sp, s)
                 : launch_traverse<BFMT, TFMT, false, false, false, KERN>(d, cd, 0.f, cfg.jac_eps, q, order, nq, D, flags, stats,
                                                                           cursor, warps, cps, sp, s);
}

template <int BFMT, int TFMT>
cudaError_t dispatch_stats(const MapDesc &d, const ClusterDesc &cd, const pndf_query *q, const uint32_t *order,
                           int64_t nq, float *D, uint32_t *flags, pndf_query_stats *stats,
                           unsigned long long *cursor, const pndf_eval_config &cfg, const SplitPlan &sp,
                           cudaStream_t s)
{
    if (cfg.jac_eps > 0.f)  // Gaussian, hierarchy mode, no cluster cut (checked by the caller)
        return stats ? launch_traverse<BFMT, TFMT, true, false, false, kKernGaussClamp>(
                           d, cd, 0.f, cfg.jac_eps, q, order, nq, D, flags, stats, cursor,
                           cfg.warps_per_cta > 0 ? cfg.warps_per_cta : 8, cfg.ctas_per_sm, sp, s)
                     : launch_traverse<BFMT, TFMT, false, false, false, kKernGaussClamp>(
                           d, cd, 0.f, cfg.jac_eps, q, order, nq, D, flags, stats, cursor,
                           cfg.warps_per_cta > 0 ? cfg.warps_per_cta : 8, cfg.ctas_per_sm, sp, s);
    if (cfg.kernel == PNDF_KERNEL_DISK)
        return dispatch_kernel<BFMT, TFMT, PNDF_KERNEL_DISK>(d, cd, q, order, nq, D, flags, stats, cursor, cfg, sp, s);
    if (cfg.kernel == PNDF_KERNEL_BOX)
        return dispatch_kernel<BFMT, TFMT, PNDF_KERNEL_BOX>(d, cd, q, order, nq, D, flags, stats, cursor, cfg, sp, s);
    return dispatch_kernel<BFMT, TFMT, PNDF_KERNEL_GAUSS>(d, cd, q, order, nq, D, flags, stats, cursor, cfg, sp, s);
}

}  // namespace

pndf_status launch_eval(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, float *D, uint32_t *flags,
                        pndf_query_stats *stats, const pndf_eval_config &cfg, cudaStream_t s)
{
    if (nq == 0) return PNDF_OK;
    const MapDesc &d = h->d;
    const bool sort = cfg.sort != 0;
    const bool split = cfg.mode == PNDF_MODE_HIERARCHY && !(cfg.tau > 0.f) && cfg.split == 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t cap = uint32_t(2 * 64 * (sms > 0 ? sms : 1) + 64);  // >= 2 x resident warps
    // scratch: cursor, split counter and work sum (padded to 256), key
    // histogram, keys, order, split markers and entries
    const size_t hist_b = sort_hist_bytes(nq);
    size_t off_hist = 256, off_keys = off_hist + hist_b;
    size_t off_order = off_keys + ((size_t(nq) * sizeof(uint32_t) + 255) & ~size_t(255));
    size_t bytes = sort ? off_order + ((size_t(nq) * sizeof(uint32_t) + 255) & ~size_t(255)) : 256;
    const size_t off_marker = bytes, off_entries = off_marker + ((size_t(nq) + 255) & ~size_t(255));
    if (split) bytes = off_entries + size_t(cap) * sizeof(SplitEntry);
    void *scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return PNDF_ERR_OOM;
    }
    char *base = static_cast<char *>(scratch);
    auto *cursor = reinterpret_cast<unsigned long long *>(base);
    SplitPlan sp{};
    if (split) {
        sp.entries = reinterpret_cast<SplitEntry *>(base + off_entries);
        sp.marker = reinterpret_cast<uint8_t *>(base + off_marker);
        sp.ctr = reinterpret_cast<unsigned long long *>(base + 8);
        sp.work = reinterpret_cast<double *>(base + 16);
        sp.cap = cap;
    }
    uint32_t *order = nullptr;
    cudaError_t e = cudaMemsetAsync(base, 0, sort ? off_keys : 256, s);
    if (e == cudaSuccess && sort) {
        order = reinterpret_cast<uint32_t *>(base + off_order);
        e = sort_launch(d, q, nq, cfg.sort, reinterpret_cast<uint32_t *>(base + off_hist),
                        reinterpret_cast<uint32_t *>(base + off_keys), order, s);
    }
    if (e == cudaSuccess && cfg.ev_begin) e = cudaEventRecord(static_cast<cudaEvent_t>(cfg.ev_begin), s);
    if (e == cudaSuccess) {
        if (d.bounds_fmt == PNDF_BOUNDS_F32)
            e = d.texel_fmt == PNDF_TEXEL_F32X2
                    ? dispatch_stats<PNDF_BOUNDS_F32, PNDF_TEXEL_F32X2>(d, h->c, q, order, nq, D, flags, stats, cursor, cfg, sp, s)
                    : dispatch_stats<PNDF_BOUNDS_F32, PNDF_TEXEL_F16X2>(d, h->c, q, order, nq, D, flags, stats, cursor, cfg, sp, s);
        else
            e = d.texel_fmt == PNDF_TEXEL_F32X2
                    ? dispatch_stats<PNDF_BOUNDS_F16_OUTWARD, PNDF_TEXEL_F32X2>(d, h->c, q, order, nq, D, flags, stats, cursor,
                                                                             cfg, sp, s)
                    : dispatch_stats<PNDF_BOUNDS_F16_OUTWARD, PNDF_TEXEL_F16X2>(d, h->c, q, order, nq, D, flags, stats, cursor,
                                                                             cfg, sp, s);
    }
    if (e == cudaSuccess && cfg.ev_end) e = cudaEventRecord(static_cast<cudaEvent_t>(cfg.ev_end), s);
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess || ef != cudaSuccess) return PNDF_ERR_CUDA;
    return PNDF_OK;
}

// ---------------------------------------------------------------------------
// Sorting a batch on its own (pndf_sort_queries).
// ---------------------------------------------------------------------------

pndf_status launch_sort(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, uint32_t *order, cudaStream_t s)
{
    if (nq == 0) return PNDF_OK;
    size_t off_keys = sort_hist_bytes(nq);
    size_t bytes = off_keys + ((size_t(nq) * sizeof(uint32_t) + 255) & ~size_t(255));
    void *scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return PNDF_ERR_OOM;
    }
    auto *hist = static_cast<uint32_t *>(scratch);
    auto *keys = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + off_keys);
    cudaError_t e = cudaMemsetAsync(hist, 0, off_keys, s);
    if (e == cudaSuccess) e = sort_launch(h->d, q, nq, PNDF_SORT_DEFAULT, hist, keys, order, s);
    cudaError_t ef = cudaFreeAsync(scratch, s);
    return (e == cudaSuccess && ef == cudaSuccess) ? PNDF_OK : PNDF_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Serving step kernel: one persistent launch over a table of segments.
//
// Table layout (device): uint32 nsegs, uint32 prefix[nsegs + 1] (prefix[0] =
// 0, prefix[i] = queries in segments 0..i-1), then the pndf_segment array at
// a 16-byte boundary.  Warps pull global work indices from one cursor; index k
// belongs to the last segment i with prefix[i] <= k.
// ---------------------------------------------------------------------------

namespace {

constexpr int kServePrefixSmem = 1025;  // prefix sums of up to 1024 segments per step in shared memory

// CLUSTER / KERN: the server's evaluation variant (the cut, the footprint
// kernel or the clamp), compiled in as for traverse_kernel.
// Segment of work index k: the last segment i with prefix[i] <= k.
__device__ __forceinline__ int serve_segment(const uint32_t *prefix, int nsegs, uint32_t k)
{
    int lo = 0, hi = nsegs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The step's division of large footprints, as for pndf_eval_batch: the work
// estimate summed over the step's queries, then the plan (which also stores
// the target w_t for the step kernel, which recomputes each query's choice).
template <int KERN>
__global__ void serve_split_work(const uint32_t *__restrict__ table, const pndf_segment *__restrict__ segs,
                                 float jac_eps, double *__restrict__ work)
{
    __shared__ double red[256];
    const int nsegs = int(table[0]);
    const uint32_t *prefix = table + 1;
    const uint32_t total = prefix[nsegs];
    double acc = 0.0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const pndf_segment &sg = segs[serve_segment(prefix, nsegs, k)];
        const int64_t j = int64_t(sg.first) + int64_t(k - prefix[&sg - segs]);
        acc += double(split_estimate(make_query(sg.q[sg.order ? int64_t(sg.order[j]) : j], KERN, jac_eps)));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(work, red[0]);
}

template <int KERN>
__global__ void serve_split_plan(const MapDesc *__restrict__ maps, const uint32_t *__restrict__ table,
                                 const pndf_segment *__restrict__ segs, float jac_eps, SplitPlan p)
{
    const float wt = split_target(p);
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.wt = wt;
    const int nsegs = int(table[0]);
    const uint32_t *prefix = table + 1;
    const uint32_t total = prefix[nsegs];
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const int i = serve_segment(prefix, nsegs, k);
        const pndf_segment &sg = segs[i];
        const int64_t j = int64_t(sg.first) + int64_t(k - prefix[i]);
        const uint32_t qi = sg.order ? sg.order[j] : uint32_t(j);
        const Query q = make_query(sg.q[qi], KERN, jac_eps);
        int level;
        uint32_t tiles;
        if (split_choice(q, maps[sg.map].L, wt, level, tiles) && !split_reserve(p, qi, i, level, tiles))
            record_status(maps[sg.map].status, &g_status_eval, PNDF_QF_OVERFLOW);
    }
}

template <int BFMT, int TFMT, bool CLUSTER, int KERN>
__global__ void __launch_bounds__(256, PNDF_TRAVERSE_MIN_CTAS)
    serve_kernel(const MapDesc *__restrict__ maps, const ClusterDesc *__restrict__ clusters, int nmaps,
                 const uint32_t *__restrict__ table, const pndf_segment *__restrict__ segs,
                 unsigned long long *__restrict__ cursor, float tau, float jac_eps, SplitPlan sp)
{
    extern __shared__ uint32_t smem[];
    __shared__ MapDesc smaps[kServeMaxMaps];
    __shared__ uint32_t sprefix[kServePrefixSmem];
    __shared__ unsigned long long s_ntiles;
    __shared__ int s_entries;
    __shared__ float s_wt;
    __shared__ uint32_t s_dest[8][3];  // per warp: segment, query, entry (-1: whole query)
    const int nsegs = int(table[0]);
    // the segment prefix sums, searched once per query, in shared memory when they fit
    const bool prefix_in_smem = nsegs < kServePrefixSmem;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(maps);
        uint32_t *dst = reinterpret_cast<uint32_t *>(smaps);
        const int words = nmaps * int(sizeof(MapDesc) / sizeof(uint32_t));
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
        if (prefix_in_smem)
            for (int i = threadIdx.x; i <= nsegs; i += blockDim.x) sprefix[i] = table[1 + i];
        if (threadIdx.x == 0) {
            // the divided queries' tiles take the first s_ntiles work indices
            int n = 0;
            unsigned long long t = 0ull;
            float wt = __int_as_float(0x7f800000);
            if (!CLUSTER && sp.entries) {
                n = int(min(__ldcg(sp.ctr) >> 40, (unsigned long long)sp.cap));
                if (n > 0) t = __ldcg(&sp.entries[n - 1].base) + __ldcg(&sp.entries[n - 1].tiles);
                wt = __ldcg(sp.wt);
            }
            s_entries = n;
            s_ntiles = t;
            s_wt = wt;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *stk = smem + warp * kWarpSmemWords;
    uint32_t *lq = stk + kStackCap;
    uint32_t *ring = lq + kLeafQ;
    float4 *hits = reinterpret_cast<float4 *>(ring + kRing + kCapRing);
    const uint32_t *prefix = prefix_in_smem ? sprefix : table + 1;
    const uint32_t total = prefix[nsegs];
    while (true) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(cursor, 1ull);
        k = __shfl_sync(kFull, k, 0);
        if (CLUSTER) {
            if (k >= total) break;
            const int i = serve_segment(prefix, nsegs, uint32_t(k));
            const pndf_segment sg = segs[i];
            const int64_t j = int64_t(sg.first) + int64_t(uint32_t(k) - prefix[i]);
            const int64_t qi = sg.order ? int64_t(sg.order[j]) : j;
            float Dv;
            uint32_t fv;
            eval_one<BFMT, TFMT, false, false, CLUSTER, KERN>(smaps[sg.map], clusters[sg.map], tau, jac_eps, sg.q[qi],
                                                               lane, stk, lq, ring, hits, Dv, fv, nullptr);
            if (lane == 0) {
                sg.D[qi] = Dv;
                if (sg.flags) sg.flags[qi] = fv;
            }
            continue;
        }
        // a tile of a divided query, or a whole query: one descent either way
        constexpr bool CLAMP = KERN == kKernGaussClamp;
        int ei = -1;
        int i;
        uint32_t qi;
        Query q;
        int e, a0, a1, c0, c1;
        if (k < s_ntiles) {
            ei = tile_entry(sp, s_entries, k);
            const SplitEntry &E = sp.entries[ei];
            i = __ldg(&E.pad);
            qi = __ldg(&E.qi);
            q = make_query(segs[i].q[qi], KERN, jac_eps);
            e = __ldg(&E.level);
            tile_range(q, smaps[segs[i].map].L, e, uint32_t(k - __ldg(&E.base)), a0, a1, c0, c1);
        } else {
            k -= s_ntiles;
            if (k >= total) break;
            i = serve_segment(prefix, nsegs, uint32_t(k));
            const int64_t j = int64_t(segs[i].first) + int64_t(uint32_t(k) - prefix[i]);
            qi = segs[i].order ? segs[i].order[j] : uint32_t(j);
            q = make_query(segs[i].q[qi], KERN, jac_eps);
            const int L = smaps[segs[i].map].L;
            if (!q.valid) {
                if (lane == 0) {
                    segs[i].D[qi] = __int_as_float(0x7fc00000);
                    if (segs[i].flags) segs[i].flags[qi] = PNDF_QF_INVALID;
                    record_status(smaps[segs[i].map].status, &g_status_eval, PNDF_QF_INVALID);
                }
                continue;
            }
            {
                int l;
                uint32_t t;
                if (split_choice(q, L, s_wt, l, t)) continue;  // evaluated as tiles
            }
            e = entry_level(q, L);
            const float sz = float(1u << e);
            node_range(q.x, q.rx, sz, 1 << (L - e), a0, a1);
            node_range(q.y, q.ry, sz, 1 << (L - e), c0, c1);
        }
        // where the result goes waits in shared memory during the descent
        if (lane == 0) {
            s_dest[warp][0] = uint32_t(i);
            s_dest[warp][1] = qi;
            s_dest[warp][2] = uint32_t(ei);
        }
        const int map = segs[i].map;
        Acc acc = {};
        acc_zero();
        eval_range<BFMT, TFMT, false, false, CLAMP>(smaps[map], kNoClusters, q, e, a0, a1, c0, c1, lane, stk, lq, ring,
                                                    hits, acc);
        unsigned long long lo, hi;
        uint32_t fl;
        warp_total<false>(acc, lo, hi, fl);
        if (lane == 0) {
            const pndf_segment &sg = segs[s_dest[warp][0]];
            const uint32_t qo = s_dest[warp][1];
            const int eo = int(s_dest[warp][2]);
            const MapDesc &md = smaps[sg.map];
            if (eo >= 0) {
                tile_finish<false>(md, sp.entries[eo], acc, lo, hi, fl, sg.D, sg.flags, nullptr);
            } else {
                sg.D[qo] = acc_value(lo, hi, fl);
                if (sg.flags) sg.flags[qo] = fl & ~kHuge;
                if (fl & PNDF_QF_OVERFLOW) record_status(md.status, &g_status_eval, PNDF_QF_OVERFLOW);
            }
        }
    }
}

template <int BFMT, int TFMT, bool CLUSTER, int KERN>
cudaError_t launch_serve_t(const ServeVariant &v, const MapDesc *maps, const ClusterDesc *clusters, int nmaps,
                           const uint32_t *table, const pndf_segment *segs, unsigned long long *cursor, int warps,
                           int ctas_per_sm, void *split, uint32_t split_cap, cudaStream_t s)
{
    auto kern = serve_kernel<BFMT, TFMT, CLUSTER, KERN>;
    int threads = warps * 32;
    size_t smem = size_t(warps) * kWarpSmemWords * sizeof(uint32_t);
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
    SplitPlan sp{};
    if (!CLUSTER && split) {
        char *b = static_cast<char *>(split);
        sp.ctr = reinterpret_cast<unsigned long long *>(b);
        sp.work = reinterpret_cast<double *>(b + 8);
        sp.wt = reinterpret_cast<float *>(b + 16);
        sp.entries = reinterpret_cast<SplitEntry *>(b + 256);
        sp.cap = split_cap;
        sp.resident_warps = sms * occ * warps;
        e = cudaMemsetAsync(split, 0, 256, s);
        if (e != cudaSuccess) return e;
        serve_split_work<KERN><<<unsigned(sms * 4), 256, 0, s>>>(table, segs, v.jac_eps, sp.work);
        serve_split_plan<KERN><<<unsigned(sms * 4), 256, 0, s>>>(maps, table, segs, v.jac_eps, sp);
    }
    kern<<<unsigned(sms * occ), threads, smem, s>>>(maps, clusters, nmaps, table, segs, cursor, v.tau, v.jac_eps, sp);
    return cudaGetLastError();
}

// Allow the variant's kernel the dynamic shared memory of `warps` warps (with
// its static tables the total passes the 48 KB a launch gets by default).
template <int BFMT, int TFMT, bool CLUSTER, int KERN>
cudaError_t serve_smem_t(int warps)
{
    return cudaFuncSetAttribute(serve_kernel<BFMT, TFMT, CLUSTER, KERN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                warps * kWarpSmemWords * int(sizeof(uint32_t)));
}

template <int BFMT, int TFMT>
cudaError_t serve_smem_v(const ServeVariant &v, int warps)
{
    if (v.tau > 0.f) return serve_smem_t<BFMT, TFMT, true, PNDF_KERNEL_GAUSS>(warps);
    if (v.jac_eps > 0.f) return serve_smem_t<BFMT, TFMT, false, kKernGaussClamp>(warps);
    if (v.kernel == PNDF_KERNEL_DISK) return serve_smem_t<BFMT, TFMT, false, PNDF_KERNEL_DISK>(warps);
    if (v.kernel == PNDF_KERNEL_BOX) return serve_smem_t<BFMT, TFMT, false, PNDF_KERNEL_BOX>(warps);
    return serve_smem_t<BFMT, TFMT, false, PNDF_KERNEL_GAUSS>(warps);
}

// The variant's instantiation: the cut (Gaussian), the plain Gaussian, disk,
// box, or the Gaussian with the Eq. 6 clamp (the server validated the mix).
template <int BFMT, int TFMT>
cudaError_t launch_serve_v(const ServeVariant &v, const MapDesc *maps, const ClusterDesc *clusters, int nmaps,
                           const uint32_t *table, const pndf_segment *segs, unsigned long long *cursor, int warps,
                           int ctas_per_sm, void *split, uint32_t split_cap, cudaStream_t s)
{
#define PNDF_SERVE(C, K)                                                                                     \
    launch_serve_t<BFMT, TFMT, C, K>(v, maps, clusters, nmaps, table, segs, cursor, warps, ctas_per_sm, split, \
                                     split_cap, s)
    if (v.tau > 0.f) return PNDF_SERVE(true, PNDF_KERNEL_GAUSS);
    if (v.jac_eps > 0.f) return PNDF_SERVE(false, kKernGaussClamp);
    if (v.kernel == PNDF_KERNEL_DISK) return PNDF_SERVE(false, PNDF_KERNEL_DISK);
    if (v.kernel == PNDF_KERNEL_BOX) return PNDF_SERVE(false, PNDF_KERNEL_BOX);
    return PNDF_SERVE(false, PNDF_KERNEL_GAUSS);
#undef PNDF_SERVE
}

}  // namespace

cudaError_t prepare_serve(int texel_fmt, int bounds_fmt, const ServeVariant &v, int warps)
{
    if (bounds_fmt == PNDF_BOUNDS_F32)
        return texel_fmt == PNDF_TEXEL_F32X2 ? serve_smem_v<PNDF_BOUNDS_F32, PNDF_TEXEL_F32X2>(v, warps)
                                             : serve_smem_v<PNDF_BOUNDS_F32, PNDF_TEXEL_F16X2>(v, warps);
    return texel_fmt == PNDF_TEXEL_F32X2 ? serve_smem_v<PNDF_BOUNDS_F16_OUTWARD, PNDF_TEXEL_F32X2>(v, warps)
                                         : serve_smem_v<PNDF_BOUNDS_F16_OUTWARD, PNDF_TEXEL_F16X2>(v, warps);
}

// Scratch of a step's division of large footprints: a 256-byte header
// (counter, work sum, target) and the entries.
uint32_t serve_split_cap()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return uint32_t(2 * 64 * (sms > 0 ? sms : 1) + 64);  // >= 2 x the resident warps
}

size_t serve_split_bytes(uint32_t cap) { return 256 + size_t(cap) * sizeof(SplitEntry); }

cudaError_t launch_serve(int texel_fmt, int bounds_fmt, const ServeVariant &v, const MapDesc *maps,
                         const ClusterDesc *clusters, int nmaps, const uint32_t *table, const pndf_segment *segs,
                         unsigned long long *cursor, int warps, int ctas_per_sm, void *split, uint32_t split_cap,
                         cudaStream_t s)
{
#define PNDF_SERVE_V(B, T) \
    launch_serve_v<B, T>(v, maps, clusters, nmaps, table, segs, cursor, warps, ctas_per_sm, split, split_cap, s)
    if (bounds_fmt == PNDF_BOUNDS_F32)
        return texel_fmt == PNDF_TEXEL_F32X2 ? PNDF_SERVE_V(PNDF_BOUNDS_F32, PNDF_TEXEL_F32X2)
                                             : PNDF_SERVE_V(PNDF_BOUNDS_F32, PNDF_TEXEL_F16X2);
    return texel_fmt == PNDF_TEXEL_F32X2 ? PNDF_SERVE_V(PNDF_BOUNDS_F16_OUTWARD, PNDF_TEXEL_F32X2)
                                         : PNDF_SERVE_V(PNDF_BOUNDS_F16_OUTWARD, PNDF_TEXEL_F16X2);
#undef PNDF_SERVE_V
}

// ---------------------------------------------------------------------------
// Allocation-free evaluation (pndf_eval_batch_noalloc).
//
// Some callers cannot allocate device memory while they evaluate: a renderer
// plugin whose host owns every device allocation and forbids others, a
// real-time thread that must not take cudaMalloc's implicit device-wide
// synchronisation or its latency, or code that budgets device memory exactly
// ahead of time.  For them the sort scratch lives in one fixed device array,
// defined here at file scope and held by every GPU that loads the library
// until the process exits.  The host never uses the array's name as an
// address: on the first call on each device, with that device current, the
// device address is looked up with cudaGetSymbolAddress and cached per
// device, keyed by the id of the context it was looked up in, so that after a
// device reset (which unloads the module with its array) the first call in the
// new context looks the address up again.
// Every call shares the array and it keeps the previous call's contents, so
// the cursor and histogram are cleared on the stream at the start of each
// call; calls whose work overlaps on the GPU (different streams, or work not
// yet complete on another stream) race on the array and must be serialised by
// the caller.
// ---------------------------------------------------------------------------

namespace {

constexpr int64_t kNoallocMaxQueries = int64_t(1) << 20;
constexpr size_t kNoallocHistOff = 256;
constexpr size_t kNoallocKeysOff = kNoallocHistOff + size_t(kKeyBins) * sizeof(uint32_t);
constexpr size_t kNoallocOrderOff = kNoallocKeysOff + size_t(kNoallocMaxQueries) * sizeof(uint32_t);
constexpr size_t kNoallocBytes = kNoallocOrderOff + size_t(kNoallocMaxQueries) * sizeof(uint32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct NoallocSlot {
    unsigned long long ctx_id;  // id of the context the address belongs to
    void *ptr;                  // device address of g_noalloc_scratch there (null: not looked up)
};

std::mutex g_noalloc_mutex;
NoallocSlot g_noalloc_slot[64] = {};

// Id of the calling thread's current context (driver entry points taken
// through the runtime, so the library links no driver library); false when
// there is none yet or the driver does not provide them.
bool current_context_id(unsigned long long *id)
{
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult r;
        return cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &r) == cudaSuccess &&
                       r == cudaDriverEntryPointSuccess
                   ? reinterpret_cast<GetCurrent>(f)
                   : nullptr;
    }();
    static GetId get_id = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult r;
        return cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &r) == cudaSuccess &&
                       r == cudaDriverEntryPointSuccess
                   ? reinterpret_cast<GetId>(f)
                   : nullptr;
    }();
    void *ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// Device address of g_noalloc_scratch on the current device: looked up on
// the first call in each context (with the device current), then cached.
cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocSlot &slot = g_noalloc_slot[dev];
    if (!have_id || !slot.ptr || slot.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!have_id) have_id = current_context_id(&id);  // the lookup made the context current
        slot.ptr = p;
        slot.ctx_id = have_id ? id : 0ull;
        if (!have_id) {  // no context id to key on: look up again next time
            *out = p;
            slot.ptr = nullptr;
            return cudaSuccess;
        }
    }
    *out = slot.ptr;
    return cudaSuccess;
}

}  // namespace

int64_t noalloc_max_queries() { return kNoallocMaxQueries; }

pndf_status launch_eval_noalloc(const pndf_hierarchy *h, const pndf_query *q, int64_t nq, float *D, uint32_t *flags,
                                cudaStream_t s)
{
    if (nq > kNoallocMaxQueries) return PNDF_ERR_CAPACITY;
    if (nq == 0) return PNDF_OK;
    void *scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return PNDF_ERR_CUDA;
    const MapDesc &d = h->d;
    pndf_eval_config cfg{PNDF_MODE_HIERARCHY, PNDF_SORT_DEFAULT, 0, 0, 0.f, PNDF_KERNEL_GAUSS, 0.f, 0, nullptr, nullptr};
    char *base = static_cast<char *>(scratch);
    auto *cursor = reinterpret_cast<unsigned long long *>(base);
    auto *hist = reinterpret_cast<uint32_t *>(base + kNoallocHistOff);
    auto *keys = reinterpret_cast<uint32_t *>(base + kNoallocKeysOff);
    auto *order = reinterpret_cast<uint32_t *>(base + kNoallocOrderOff);
    // cursor and histogram start at zero
    cudaError_t e = cudaMemsetAsync(base, 0, kNoallocHistOff + sort_hist_bytes(nq), s);
    if (e != cudaSuccess) return PNDF_ERR_CUDA;
    e = sort_launch(d, q, nq, cfg.sort, hist, keys, order, s);
    if (e != cudaSuccess) return PNDF_ERR_CUDA;
    if (d.bounds_fmt == PNDF_BOUNDS_F32)
        e = d.texel_fmt == PNDF_TEXEL_F32X2
                ? dispatch_stats<PNDF_BOUNDS_F32, PNDF_TEXEL_F32X2>(d, h->c, q, order, nq, D, flags, nullptr, cursor, cfg, SplitPlan{}, s)
                : dispatch_stats<PNDF_BOUNDS_F32, PNDF_TEXEL_F16X2>(d, h->c, q, order, nq, D, flags, nullptr, cursor, cfg, SplitPlan{}, s);
    else
        e = d.texel_fmt == PNDF_TEXEL_F32X2
                ? dispatch_stats<PNDF_BOUNDS_F16_OUTWARD, PNDF_TEXEL_F32X2>(d, h->c, q, order, nq, D, flags, nullptr, cursor,
                                                                         cfg, SplitPlan{}, s)
                : dispatch_stats<PNDF_BOUNDS_F16_OUTWARD, PNDF_TEXEL_F16X2>(d, h->c, q, order, nq, D, flags, nullptr, cursor,
                                                                         cfg, SplitPlan{}, s);
    return e == cudaSuccess ? PNDF_OK : PNDF_ERR_CUDA;
}

namespace {
__global__ void take_eval_word(unsigned int *out) { *out = atomicExch(&g_status_eval, 0u); }
}  // namespace

cudaError_t take_status_eval(unsigned int *out, cudaStream_t s)
{
    take_eval_word<<<1, 1, 0, s>>>(out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pndf
