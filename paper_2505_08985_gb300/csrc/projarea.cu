// Analytic projected area P(w) of a footprint (Sec. 4.3, Eq. 9-11, App. B).
//
//   P(w) = sum over footprint triangles T of k_r(T) / |cross(T)| * V_T(w),
//   V_T(w) = integral over n+(T) of (w . m~) / m~_z dm,
// where n+(T) is the part of the normal triangle whose normals see w, k_r(T)
// the kernel at T's uv centroid (cut where q > 16), cross(T) = (n_b - n_a) x
// (n_c - n_a).  Every triangle in the footprint is integrated (no pruning:
// every visible triangle contributes).
//
// Per triangle:
//  * all three vertices see w  =>  the whole triangle does (the visible region,
//    a right half-disk joined to a left half-ellipse, is convex; App. B), and
//    V_T = w_z A + w_x Wx + w_y Wy with Wx = -oint m~_z dm_y, Wy = oint m~_z
//    dm_x (Green's theorem on d(-m~_z)/dm_x = m_x/m~_z).  Along an edge the
//    mean of m~_z is the arc-area formula of App. B; it is evaluated in a
//    cancellation-free form (the asin difference as one atan2 of exact
//    products), so no rotation is needed and the 1/|cross| division keeps
//    FP32 accuracy for small triangles.  Small slivers (longest edge^2 below
//    1e-4 and aspect above 2) take the 3-point edge-midpoint rule on
//    max(m~.w, 0)/m~_z instead, exact for quadratics.
//  * no vertex sees w and the triangle stays clear of the visibility
//    boundary: exactly 0 (Alg. 1 drops every edge).
//  * otherwise (partly visible, slivers of aspect above 2000, normals
//    collapsed onto a segment): the general path of visible.cuh in FP64 (the
//    clip of Alg. 1 as a line-circle intersection in a scaled frame, Eq. 11's
//    boundary integral as a corner fan plus chord and arc excesses, and the
//    segment form of Eq. 13 in closed form), deferred and evaluated 32
//    triangles at a time so that it runs lane-dense.
//
// Work decomposition: each request's footprint is cut into bands of kBand quad
// rows; one warp integrates one band (lane = quad column, two triangles per
// lane), compensated sums are reduced across the warp and stored per band;
// a second kernel adds a request's bands in fixed order, so results do not
// depend on scheduling or on which other requests share the launch.
#include "area_step.cuh"
#include "ggx.cuh"
#include "visible.cuh"

namespace pndf {

__device__ unsigned int g_status_projarea;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBand = 8;                 // quad rows per work item

__device__ __forceinline__ float dop(float a, float b, float c, float d)
{
    float w = c * d;
    float e = fmaf(-c, d, w);
    float f = fmaf(a, b, -w);
    return f + e;
}

__device__ __forceinline__ float zof(float2 p)
{
    return sqrtf(fmaxf(0.f, 1.f - fmaf(p.x, p.x, p.y * p.y)));
}

// phi(t) = t - sin t, by its Taylor series for small |t| (no cancellation).
__device__ __forceinline__ float phi_small(float t)
{
    if (fabsf(t) < 0.25f) {
        float t2 = t * t;
        return t * t2 * (1.f / 6.f) * (1.f - t2 * (1.f / 20.f) * (1.f - t2 * (1.f / 42.f) * (1.f - t2 * (1.f / 72.f))));
    }
    return t - sinf(t);
}

// Curvature part H of the mean of m~_z = sqrt(1 - |m|^2) along p0 -> p1, over
// its trapezoid value (z0 + z1)/2.  With d the unit direction, u the abscissa
// along the line (u1 = u0 + L) and r^2 = 1 - s^2 = z0^2 + u0^2 (s the line's
// distance to the origin), the arc-area formula of App. B gives
//   L * mean = (1/2)[u z]_{u0}^{u1} + (r^2/2)(asin(u1/r) - asin(u0/r)),
// so L * H = (r^2/2)(dth - sin dth) with dth the asin difference, which is
// atan2(X, Y), X = u1 z0 - u0 z1 = L (r^2 + z0 z1 + u0 u1) / (z0 + z1),
// Y = z0 z1 + u0 u1 (both free of cancellation).
__device__ __forceinline__ float edge_curv(float2 p0, float z0, float2 p1, float z1)
{
    float ex = p1.x - p0.x, ey = p1.y - p0.y;
    float L2 = fmaf(ex, ex, ey * ey);
    if (L2 == 0.f) return 0.f;
    float L = sqrtf(L2);
    float inv = 1.f / L;
    float u0 = fmaf(ex, p0.x, ey * p0.y) * inv;
    float u1 = u0 + L;
    float r2 = fmaf(z0, z0, u0 * u0);
    float Y = fmaf(z0, z1, u0 * u1);
    float X = L * (r2 + Y) / (z0 + z1);
    return 0.5f * r2 * phi_small(atan2f(X, Y)) * inv;
}

// z(q) - z(p) for z = sqrt(1 - |m|^2), from (|p|^2 - |q|^2) / (z(p) + z(q)).
__device__ __forceinline__ float zdiff(float2 p, float zp, float2 q, float zq)
{
    return -fmaf(q.x - p.x, q.x + p.x, (q.y - p.y) * (q.y + p.y)) / (zp + zq);
}

struct Dir {
    float wx, wy, wz;  // unit direction
    float c, s, wr;    // rotation to w_y = 0: (c, s) = w_xy / |w_xy|, wr = |w_xy|
};

// Unit direction from the caller's (unit to single precision) vector.
__device__ __forceinline__ Dir make_dir_f(float wx, float wy, float wz)
{
    Dir w;
    const float n = sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
    w.wx = wx / n;
    w.wy = wy / n;
    w.wz = wz / n;
    w.wr = sqrtf(fmaf(w.wx, w.wx, w.wy * w.wy));
    w.c = w.wr > 0.f ? w.wx / w.wr : 1.f;
    w.s = w.wr > 0.f ? w.wy / w.wr : 0.f;
    return w;
}

// V_T / |cross| on the general path (visible.cuh, FP64): partly visible
// triangles, long slivers, and triangles whose normals collapsed onto a
// segment (|cross| < 1e-12: the segment form of Eq. 13).
__device__ __noinline__ float slow_ratio(float2 a, float2 b, float2 c, const Dir &wf)
{
    const vis::DirD w = vis::make_dir(wf.wx, wf.wy, wf.wz);
    const double cr = (double(b.x) - double(a.x)) * (double(c.y) - double(a.y)) -
                      (double(b.y) - double(a.y)) * (double(c.x) - double(a.x));
    if (fabs(cr) < 1e-12) return float(vis::collapsed_visible(a.x, a.y, b.x, b.y, c.x, c.y, w));
    return float(vis::tri_visible<double>(a.x, a.y, b.x, b.y, c.x, c.y, w));
}

// Squared distance from the origin to segment p -> q.
__device__ __forceinline__ float seg_dist2(float px, float py, float qx, float qy)
{
    float vx = qx - px, vy = qy - py;
    float L2 = fmaf(vx, vx, vy * vy);
    float t = L2 > 0.f ? fminf(fmaxf(-fmaf(px, vx, py * vy) / L2, 0.f), 1.f) : 0.f;
    float dx = fmaf(t, vx, px), dy = fmaf(t, vy, py);
    return fmaf(dx, dx, dy * dy);
}

// True when the triangle provably sees nothing of w: in the frame rotated so
// w_y = 0 all three vertices have m_x < 0 (the visible part there is the
// half-ellipse (m_x / w_z)^2 + m_y^2 <= 1) and the triangle stays clear of
// that ellipse (distance > 1 from the origin after scaling m_x by 1 / w_z,
// with a margin for FP32 rounding).  Alg. 1 drops every edge of such a
// triangle, so its integral is exactly 0.
__device__ __forceinline__ bool invisible_and_clear(float2 a, float2 b, float2 c, const Dir &w)
{
    float ax = fmaf(w.c, a.x, w.s * a.y), bx = fmaf(w.c, b.x, w.s * b.y), cx = fmaf(w.c, c.x, w.s * c.y);
    if (!(ax < 0.f && bx < 0.f && cx < 0.f)) return false;
    float ay = fmaf(-w.s, a.x, w.c * a.y), by = fmaf(-w.s, b.x, w.c * b.y), cy = fmaf(-w.s, c.x, w.c * c.y);
    float iz = 1.f / w.wz;
    ax *= iz;
    bx *= iz;
    cx *= iz;
    // the origin must not lie inside the scaled triangle
    float o0 = dop(bx - ax, -ay, by - ay, -ax), o1 = dop(cx - bx, -by, cy - by, -bx), o2 = dop(ax - cx, -cy, ay - cy, -cx);
    if ((o0 >= 0.f && o1 >= 0.f && o2 >= 0.f) || (o0 <= 0.f && o1 <= 0.f && o2 <= 0.f)) return false;
    float d2 = fminf(seg_dist2(ax, ay, bx, by), fminf(seg_dist2(bx, by, cx, cy), seg_dist2(cx, cy, ax, ay)));
    return d2 > 1.0045f;  // (1 + 2.25e-3)^2
}

// V_T / |cross| for one triangle in FP32 when that is accurate: returns false
// when the triangle needs the FP64 path (partially visible, long sliver,
// collapsed), which the caller defers and batches.
__device__ __forceinline__ bool tri_ratio_fast(float2 a, float za, float2 b, float zb, float2 c, float zc,
                                               const Dir &w, float &out)
{
    float va = fmaf(w.wx, a.x, fmaf(w.wy, a.y, w.wz * za));
    float vb = fmaf(w.wx, b.x, fmaf(w.wy, b.y, w.wz * zb));
    float vc = fmaf(w.wx, c.x, fmaf(w.wy, c.y, w.wz * zc));
    float2 ab = make_float2(b.x - a.x, b.y - a.y), ac = make_float2(c.x - a.x, c.y - a.y);
    float2 bc = make_float2(c.x - b.x, c.y - b.y);
    float cr = dop(ab.x, ac.y, ab.y, ac.x);
    float P2 = fmaxf(fmaf(ab.x, ab.x, ab.y * ab.y), fmaxf(fmaf(ac.x, ac.x, ac.y * ac.y), fmaf(bc.x, bc.x, bc.y * bc.y)));
    if (!(va >= 0.f && vb >= 0.f && vc >= 0.f)) {
        // partially visible triangles take the FP64 path: when most of a
        // footprint is shadowed P itself is tiny, and FP32 clipping (roots of
        // nearly tangent edges, arcs) would dominate its relative error
        out = 0.f;
        return invisible_and_clear(a, b, c, w);
    }
    if (P2 == 0.f) {  // all three normals equal
        out = 0.5f * (w.wz + fmaf(w.wx, a.x, w.wy * a.y) / za);
        return true;
    }
    // The boundary form below has FP32 error about 1.5 eps P^2 / |cross|.
    if (P2 > 2.0f * fabsf(cr)) {
        if (P2 < 1e-4f) {
            // small sliver: 3-point edge-midpoint rule (exact for quadratics) on
            // the mean of (w . m~)/m~_z; V / |cross| = mean / 2
            float2 m0 = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
            float2 m1 = make_float2(0.5f * (b.x + c.x), 0.5f * (b.y + c.y));
            float2 m2 = make_float2(0.5f * (c.x + a.x), 0.5f * (c.y + a.y));
            float z0 = zof(m0), z1 = zof(m1), z2 = zof(m2);
            float f0 = fmaf(w.wx, m0.x, w.wy * m0.y) / z0;
            float f1 = fmaf(w.wx, m1.x, w.wy * m1.y) / z1;
            float f2 = fmaf(w.wx, m2.x, w.wy * m2.y) / z2;
            out = 0.5f * w.wz + (f0 + f1 + f2) * (1.f / 6.f);
            return true;
        }
        if (P2 > 2000.0f * fabsf(cr)) return false;  // long sliver or collapsed: FP64
    }
    // Fully visible: V = w_z A + w_x Wx + w_y Wy, Wx = -oint m~_z dm_y,
    // Wy = oint m~_z dm_x.  With the edge mean of m~_z split into its
    // trapezoid value and the curvature part H, the trapezoid sums collapse to
    // 2x2 determinants of vertex differences in (x, z) and (y, z).
    float dzab = zdiff(a, za, b, zb), dzac = zdiff(a, za, c, zc);
    float dety = dop(ab.y, dzac, ac.y, dzab);
    float detx = dop(ab.x, dzac, ac.x, dzab);
    float hab = edge_curv(a, za, b, zb), hbc = edge_curv(b, zb, c, zc), hca = edge_curv(c, zc, a, za);
    float Wx = 0.5f * dety - (hab * ab.y + hbc * bc.y - hca * ac.y);
    float Wy = -0.5f * detx + (hab * ab.x + hbc * bc.x - hca * ac.x);
    // orientation-following integrals over the signed cross = the
    // counter-clockwise value over |cross|
    out = 0.5f * w.wz + fmaf(w.wx, Wx, w.wy * Wy) / cr;
    return true;
}

struct Req {
    float x, y, ia, ib, ic, norm, ry;
    int j0, j1, i0, i1;
    bool valid;
};

__device__ __forceinline__ Req make_req(const pndf_query &r, int n)
{
    Req q;
    float det = r.sxx * r.syy - r.sxy * r.sxy;
    q.valid = (r.sxx > 0.f) && (r.syy > 0.f) && (det > 0.f) && isfinite(det) && isfinite(r.x) && isfinite(r.y);
    q.x = r.x;
    q.y = r.y;
    float inv = 1.f / det;
    q.ia = r.syy * inv;
    q.ib = -r.sxy * inv;
    q.ic = r.sxx * inv;
    q.norm = 1.f / (2.f * kPi * sqrtf(det));
    float rx = 4.f * sqrtf(r.sxx) * (1.f + 1e-5f) + 1e-6f;
    q.ry = 4.f * sqrtf(r.syy) * (1.f + 1e-5f) + 1e-6f;
    // quads whose centroid (i + 1/3 or 2/3) can lie in the 4-sigma box
    // clamped in float first so no int conversion can overflow
    float fi0 = fmaxf(floorf(r.x - rx) - 1.f, 0.f), fi1 = fminf(ceilf(r.x + rx), float(n - 2));
    float fj0 = fmaxf(floorf(r.y - q.ry) - 1.f, 0.f), fj1 = fminf(ceilf(r.y + q.ry), float(n - 2));
    bool empty = !(fi0 <= fi1) || !(fj0 <= fj1);
    q.i0 = empty ? 0 : int(fi0);
    q.i1 = empty ? -1 : int(fi1);
    q.j0 = empty ? 0 : int(fj0);
    q.j1 = empty ? -1 : int(fj1);
    if (!q.valid || q.i0 > q.i1 || q.j0 > q.j1) {
        q.i1 = q.i0 - 1;
        q.j1 = q.j0 - 1;
    }
    return q;
}

__device__ __forceinline__ float wq(const Req &q, float dx, float dy)
{
    return fmaf(q.ia * dx, dx, fmaf(2.f * q.ib * dx, dy, q.ic * dy * dy));
}

template <int TFMT>
__device__ __forceinline__ float2 texel(const MapDesc &d, int i, int j)
{
    size_t idx = size_t(j) * d.n + i;
    if (TFMT == PNDF_TEXEL_F32X2) return __ldg(reinterpret_cast<const float2 *>(d.texels) + idx);
    return __half22float2(__ldg(reinterpret_cast<const __half2 *>(d.texels) + idx));
}

// Ring of triangles deferred to the FP64 path, per warp: (i << 15) | (j << 1)
// | tri and the triangle's kernel weight; processed 32 at a time so the slow
// path runs with every lane busy.
constexpr int kDefer = 128;

// Lane's deferred triangle (ring slot head + lane): kernel weight times the
// FP64 value of V_T / |cross| (tri 0 = (u0, u1, u2), tri 1 = (u3, u2, u1)).
template <int TFMT>
__device__ __forceinline__ float deferred_value(const MapDesc &d, const Dir &w, const uint32_t *dq_id,
                                                const float *dq_w, uint32_t head, int lane)
{
    uint32_t slot = (head + uint32_t(lane)) & (kDefer - 1);
    uint32_t id = dq_id[slot];
    int i = int(id >> 15), j = int((id >> 1) & 0x3fffu), tri = int(id & 1u);
    float2 a = texel<TFMT>(d, i + tri, j + tri);
    float2 b = texel<TFMT>(d, i + 1 - tri, j + tri);
    float2 c = texel<TFMT>(d, i + tri, j + 1 - tri);
    return dq_w[slot] * slow_ratio(a, b, c, w);
}

__global__ void pa_bands(MapDesc d, const pndf_query *__restrict__ qs, int64_t k0, int cnt, uint32_t *__restrict__ nb)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    Req q = make_req(qs[k0 + t], d.n);
    int rows = q.j1 - q.j0 + 1;
    nb[t] = rows > 0 ? uint32_t((rows + kBand - 1) / kBand) : 0u;
}

// exclusive scan of cnt (<= 65536) values in place, one CTA of 1024 threads;
// total goes to nb[cnt]
__device__ __forceinline__ void scan_bands(uint32_t *__restrict__ nb, int cnt)
{
    __shared__ uint32_t part[1024];
    const int per = (cnt + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    uint32_t sum = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < cnt) sum += nb[b0 + i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - sum;
    for (int i = 0; i < per; ++i) {
        if (b0 + i < cnt) {
            uint32_t v = nb[b0 + i];
            nb[b0 + i] = run;
            run += v;
        }
    }
    if (threadIdx.x == 1023) nb[cnt] = part[1023];
}

__global__ void __launch_bounds__(1024) pa_scan(uint32_t *__restrict__ nb, int cnt) { scan_bands(nb, cnt); }

// Band `band` (kBand quad rows) of request (q, w) on map d, integrated by one
// warp (lane = quad column, both triangles; the FP64 triangles deferred into
// the warp's ring dq_id / dq_w and evaluated 32 at a time); returns the
// compensated sum and its correction, reduced to lane 0 in a fixed order.
template <int TFMT>
__device__ __forceinline__ float2 integrate_band(const MapDesc &d, const Req &q, const Dir &w, int band, int lane,
                                                 uint32_t *dq_id, float *dq_w)
{
    const unsigned lt = (1u << lane) - 1u;
    const int jb0 = q.j0 + band * kBand, jb1 = min(q.j1, jb0 + kBand - 1);
    float s = 0.f, c = 0.f;
    uint32_t head = 0;
    int nd = 0;  // deferred triangles waiting in the ring (warp-uniform)
    for (int j = jb0; j <= jb1; ++j) {
        const float dyl = (float(j) - q.y) + (1.f / 3.f), dyu = (float(j) - q.y) + (2.f / 3.f);
        for (int ib = q.i0; ib <= q.i1; ib += 32) {
            const int i = ib + lane;
            float v[2] = {0.f, 0.f}, kw[2] = {0.f, 0.f};
            bool dfr[2] = {false, false};
            if (i <= q.i1) {
                const float dxl = (float(i) - q.x) + (1.f / 3.f), dxu = (float(i) - q.x) + (2.f / 3.f);
                const float ql = wq(q, dxl, dyl), qu = wq(q, dxu, dyu);
                if (ql <= kQCut || qu <= kQCut) {
                    // one copy of the triangle path for both triangles (tri 0 =
                    // (u0, u1, u2), tri 1 = (u3, u2, u1)): unrolled, the kernel
                    // stalled on instruction fetch (516 ms against 386 ms); the
                    // quad's four texels are loaded together
                    const float2 n1 = texel<TFMT>(d, i + 1, j), n2 = texel<TFMT>(d, i, j + 1);
                    const float2 n0 = texel<TFMT>(d, i, j), n3 = texel<TFMT>(d, i + 1, j + 1);
                    const float z1 = zof(n1), z2 = zof(n2);
#pragma unroll 1
                    for (int k = 0; k < 2; ++k) {
                        const float qk = k ? qu : ql;
                        if (qk > kQCut) continue;
                        const float2 na = k ? n3 : n0;
                        const float2 nb = k ? n2 : n1, nc = k ? n1 : n2;
                        const float zb = k ? z2 : z1, zc = k ? z1 : z2;
                        float r;
                        const float kk = q.norm * expf(-0.5f * qk);
                        const bool ok = tri_ratio_fast(na, zof(na), nb, zb, nc, zc, w, r);
                        if (k) {
                            kw[1] = kk;
                            v[1] = ok ? kk * r : 0.f;
                            dfr[1] = !ok;
                        } else {
                            kw[0] = kk;
                            v[0] = ok ? kk * r : 0.f;
                            dfr[0] = !ok;
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                float tt = s + v[k];
                c += fabsf(s) >= fabsf(v[k]) ? (s - tt) + v[k] : (v[k] - tt) + s;
                s = tt;
                // queue the triangles that need the FP64 path
                unsigned m = __ballot_sync(kFull, dfr[k]);
                if (dfr[k]) {
                    uint32_t pos = (head + uint32_t(nd) + __popc(m & lt)) & (kDefer - 1);
                    dq_id[pos] = (uint32_t(i) << 15) | (uint32_t(j) << 1) | uint32_t(k);
                    dq_w[pos] = kw[k];
                }
                nd += __popc(m);
            }
            __syncwarp();
            while (nd >= 32) {
                float val = deferred_value<TFMT>(d, w, dq_id, dq_w, head, lane);
                float tt = s + val;
                c += fabsf(s) >= fabsf(val) ? (s - tt) + val : (val - tt) + s;
                s = tt;
                head += 32;
                nd -= 32;
                __syncwarp();
            }
        }
    }
    if (nd > 0) {
        float val = lane < nd ? deferred_value<TFMT>(d, w, dq_id, dq_w, head, lane) : 0.f;
        float tt = s + val;
        c += fabsf(s) >= fabsf(val) ? (s - tt) + val : (val - tt) + s;
        s = tt;
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float so = __shfl_down_sync(kFull, s, o), co = __shfl_down_sync(kFull, c, o);
        float tt = s + so;
        float err = fabsf(s) >= fabsf(so) ? (s - tt) + so : (so - tt) + s;
        s = tt;
        c += co + err;
    }
    return make_float2(s, c);
}

// Eight CTAs per SM (32 registers, some spilled): 285 ms against 319 ms at
// six and 516 ms at two for 1,024 requests on a 4096^2 mixed map; the warps
// that wait on the FP64 path need company to keep the SM issuing.
template <int TFMT>
__global__ void __launch_bounds__(256, 8) pa_items(MapDesc d, const pndf_query *__restrict__ qs,
                                               const float *__restrict__ omega, int64_t k0, int cnt,
                                               const uint32_t *__restrict__ off, float2 *__restrict__ part,
                                               unsigned int *__restrict__ cursor)
{
    __shared__ uint32_t dq_id_s[8][kDefer];
    __shared__ float dq_w_s[8][kDefer];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *dq_id = dq_id_s[warp];
    float *dq_w = dq_w_s[warp];
    const uint32_t total = off[cnt];
    while (true) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(cursor, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= total) break;
        // request owning this item: last t with off[t] <= it
        int lo = 0, hi = cnt - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= it)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int t = lo;
        const Req q = make_req(qs[k0 + t], d.n);
        const Dir w = make_dir_f(omega[3 * (k0 + t)], omega[3 * (k0 + t) + 1], omega[3 * (k0 + t) + 2]);
        const float2 v = integrate_band<TFMT>(d, q, w, int(it - off[t]), lane, dq_id, dq_w);
        if (lane == 0) part[it] = v;
    }
}

// A request's P from its bands [b0, b1): one warp, fixed-order compensated
// sum (lane 0 gets the value); NaN for an invalid covariance.
__device__ __forceinline__ bool request_valid(const pndf_query &r)
{
    const float det = r.sxx * r.syy - r.sxy * r.sxy;
    return (r.sxx > 0.f) && (r.syy > 0.f) && (det > 0.f) && isfinite(det) && isfinite(r.x) && isfinite(r.y);
}

__device__ __forceinline__ float reduce_bands(const float2 *__restrict__ part, uint32_t b0, uint32_t b1, int lane)
{
    float s = 0.f, c = 0.f;
    for (uint32_t b = b0 + lane; b < b1; b += 32) {
        float2 p = part[b];
        float tt = s + p.x;
        c += (fabsf(s) >= fabsf(p.x) ? (s - tt) + p.x : (p.x - tt) + s) + p.y;
        s = tt;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float so = __shfl_down_sync(kFull, s, o), co = __shfl_down_sync(kFull, c, o);
        float tt = s + so;
        float err = fabsf(s) >= fabsf(so) ? (s - tt) + so : (so - tt) + s;
        s = tt;
        c += co + err;
    }
    return s + c;
}

// one warp per request: fixed-order sum of its bands
__global__ void pa_reduce(const pndf_query *__restrict__ qs, int64_t k0, int cnt, const uint32_t *__restrict__ off,
                          const float2 *__restrict__ part, float *__restrict__ P, unsigned int *hier_status)
{
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= cnt) return;
    const float v = reduce_bands(part, off[t], off[t + 1], lane);
    if (lane == 0) {
        const bool valid = request_valid(qs[k0 + t]);
        if (!valid) record_status(hier_status, &g_status_projarea, PNDF_QF_INVALID);
        P[k0 + t] = valid ? v : __int_as_float(0x7fc00000);
    }
}

// ---- projected-area requests inside a serving step (area_step.cuh) ----

constexpr int kStepMaxMaps = kServeMaxMaps;

__global__ void area_step_bands(const MapDesc *__restrict__ maps, const uint32_t *__restrict__ count,
                                const AreaReq *__restrict__ areq, uint32_t *__restrict__ nb)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= int(*count)) return;
    const AreaReq a = areq[t];
    const Req q = make_req(*a.q, maps[a.map].n);
    const int rows = q.j1 - q.j0 + 1;
    nb[t] = rows > 0 ? uint32_t((rows + kBand - 1) / kBand) : 0u;
}

__global__ void __launch_bounds__(1024) area_step_scan(const uint32_t *__restrict__ count, uint32_t *__restrict__ nb)
{
    scan_bands(nb, int(*count));
}

template <int TFMT>
__global__ void __launch_bounds__(256, 8) area_step_items(const MapDesc *__restrict__ maps, int nmaps,
                                                      const uint32_t *__restrict__ count,
                                                      const AreaReq *__restrict__ areq,
                                                      const uint32_t *__restrict__ off, float2 *__restrict__ part,
                                                      unsigned int *__restrict__ cursor)
{
    __shared__ uint32_t dq_id_s[8][kDefer];
    __shared__ float dq_w_s[8][kDefer];
    __shared__ MapDesc smaps[kStepMaxMaps];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(maps);
        uint32_t *dst = reinterpret_cast<uint32_t *>(smaps);
        const int words = nmaps * int(sizeof(MapDesc) / sizeof(uint32_t));
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *dq_id = dq_id_s[warp];
    float *dq_w = dq_w_s[warp];
    const int cnt = int(*count);
    if (cnt == 0) return;
    const uint32_t total = off[cnt];
    while (true) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(cursor, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= total) break;
        int lo = 0, hi = cnt - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= it)
                lo = mid;
            else
                hi = mid - 1;
        }
        const AreaReq a = areq[lo];
        const MapDesc &d = smaps[a.map];
        const Req q = make_req(*a.q, d.n);
        const Dir w = make_dir_f(a.w[0], a.w[1], a.w[2]);
        const float2 v = integrate_band<TFMT>(d, q, w, int(it - off[lo]), lane, dq_id, dq_w);
        if (lane == 0) part[it] = v;
    }
}

__global__ void area_step_reduce(const MapDesc *__restrict__ maps, const uint32_t *__restrict__ count,
                                 const AreaReq *__restrict__ areq, const uint32_t *__restrict__ off,
                                 const float2 *__restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= int(*count)) return;
    const float v = reduce_bands(part, off[t], off[t + 1], lane);
    if (lane == 0) {
        const AreaReq a = areq[t];
        const bool valid = request_valid(*a.q);
        if (!valid) record_status(maps[a.map].status, &g_status_projarea, PNDF_QF_INVALID);
        *a.out = valid ? v : __int_as_float(0x7fc00000);
    }
}

// ---- GGX projected-area fit per mip node (Eq. 12) ----
//
// P'(w) = (w_z + sqrt(w_z^2 + w^T Omega w)) / 2 (Eq. 12, parentheses
// restored).  A node is box-filtered over its own quads, so its projected
// area is P(w) = 4^-l sum over its triangles of V_T / |cross| (Eq. 9-11,
// exact for the box); the fit takes P at the 16 fit directions, forms a_k =
// (2 P_k - w_z)^2 - w_z^2 = w^T Omega w and solves the 3 x 3 normal
// equations in FP64.  Leaf blocks are summed by one warp each (lane =
// triangle, FP32 per-triangle values with the FP64 path where needed); a
// parent's P is the mean of its children's.

struct GgxDirs {
    Dir w[kGgxDirs];
};

__device__ bool ggx_fit(const float *P, const GgxDirs &dirs, float4 &out)
{
    double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, r[3] = {0, 0, 0};
    for (int k = 0; k < kGgxDirs; ++k) {
        const double wx = dirs.w[k].wx, wy = dirs.w[k].wy, wz = dirs.w[k].wz;
        const double t = 2.0 * double(P[k]) - wz;
        const double a = t * t - wz * wz;
        const double row[3] = {wx * wx, 2.0 * wx * wy, wy * wy};
        for (int p = 0; p < 3; ++p) {
            r[p] += row[p] * a;
            for (int q = 0; q < 3; ++q) A[p][q] += row[p] * row[q];
        }
    }
    // Cholesky of the symmetric positive definite 3 x 3 system
    double L[3][3];
    for (int j = 0; j < 3; ++j) {
        double dd = A[j][j];
        for (int k = 0; k < j; ++k) dd -= L[j][k] * L[j][k];
        if (!(dd > 0.0)) return false;
        dd = sqrt(dd);
        L[j][j] = dd;
        for (int i = j + 1; i < 3; ++i) {
            double v = A[i][j];
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v / dd;
        }
    }
    double y[3], x[3];
    for (int i = 0; i < 3; ++i) {
        double v = r[i];
        for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
        y[i] = v / L[i][i];
    }
    for (int i = 2; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < 3; ++k) v -= L[k][i] * x[k];
        x[i] = v / L[i][i];
    }
    out = make_float4(float(x[0]), float(x[1]), float(x[2]), 0.f);
    return true;
}

__device__ __forceinline__ bool ggx_node_inside(const MapDesc &d, int l, uint32_t m)
{
    const int64_t a = int64_t(1) << l;
    return a * (compact1by1(m) + 1) <= int64_t(d.n) - 1 && a * (compact1by1(m >> 1) + 1) <= int64_t(d.n) - 1;
}

// Vertices of triangle `lane` of leaf block (i0, j0) (lane = 2 quad + tri,
// quads row-major in the 4 x 4 block; tri 0 = (u0, u1, u2), 1 = (u3, u2, u1)).
template <int TFMT>
__device__ __forceinline__ void leaf_triangle(const MapDesc &d, int i0, int j0, int lane, float2 &a, float2 &b,
                                              float2 &c)
{
    const int q = lane >> 1, tri = lane & 1;
    const int i = i0 + (q & 3), j = j0 + (q >> 2);
    a = texel<TFMT>(d, i + tri, j + tri);
    b = texel<TFMT>(d, i + 1 - tri, j + tri);
    c = texel<TFMT>(d, i + tri, j + 1 - tri);
}

// One warp per leaf block (Morton index): P at the fit directions (NaN when
// the block has a quad outside the map) and the block's fit.  Each lane
// evaluates its triangle at every direction in FP32 where that is accurate;
// the (triangle, direction) pairs that need the FP64 path are listed and
// spread over the warp 32 at a time, so the slow path runs lane-dense.  The
// per-direction sums then run in the same fixed order either way.
constexpr int kGgxLeafWarps = 8;
static_assert(kGgxDirs <= 16, "a listed pair packs the direction in 4 bits");

// Eight CTAs per SM: 68 ms against 75 ms at the register-limited two for a
// 4096^2 map (FP64 pairs dominate; more warps keep the FP64 pipe fed).
template <int TFMT>
__global__ void __launch_bounds__(32 * kGgxLeafWarps, 8) ggx_leaf(MapDesc d, GgxDirs dirs,
                                                               float *__restrict__ P, float4 *__restrict__ omega,
                                                               uint32_t nleaf)
{
    __shared__ float r_s[kGgxLeafWarps][kGgxDirs][32];
    __shared__ uint16_t item_s[kGgxLeafWarps][kGgxDirs * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (m >= nleaf) return;
    float *Pm = P + size_t(m) * kGgxDirs;
    if (!ggx_node_inside(d, kLeafLevel, m)) {
        if (lane < kGgxDirs) Pm[lane] = __int_as_float(0x7fc00000);
        if (lane == 0) omega[m] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        return;
    }
    float(*rs)[32] = r_s[warp];
    uint16_t *items = item_s[warp];
    const int i0 = int(compact1by1(m)) * kLeafQuads, j0 = int(compact1by1(m >> 1)) * kLeafQuads;
    float2 na, nb, nc;
    leaf_triangle<TFMT>(d, i0, j0, lane, na, nb, nc);
    const float za = zof(na), zb = zof(nb), zc = zof(nc);
    uint32_t need = 0;  // bit k: direction k needs the FP64 path
    for (int k = 0; k < kGgxDirs; ++k) {
        float r;
        if (tri_ratio_fast(na, za, nb, zb, nc, zc, dirs.w[k], r))
            rs[k][lane] = r;
        else
            need |= 1u << k;
    }
    // list the FP64 pairs (lane-major) and evaluate them 32 at a time
    const int cnt = __popc(need);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    for (int p = incl - cnt; need; need &= need - 1) items[p++] = uint16_t((lane << 4) | (__ffs(need) - 1));
    __syncwarp();
    for (int t0 = 0; t0 < total; t0 += 32) {
        if (t0 + lane < total) {
            const int it = items[t0 + lane], src = it >> 4, k = it & 15;
            float2 a, b, c;
            leaf_triangle<TFMT>(d, i0, j0, src, a, b, c);
            rs[k][src] = slow_ratio(a, b, c, dirs.w[k]);
        }
    }
    __syncwarp();
    for (int k = 0; k < kGgxDirs; ++k) {
        float r = rs[k][lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(kFull, r, off);  // fixed order
        if (lane == 0) Pm[k] = r * (1.0f / float(kLeafQuads * kLeafQuads));
    }
    __syncwarp();
    if (lane == 0) {
        float4 o;
        if (!ggx_fit(Pm, dirs, o)) o = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        omega[m] = o;
    }
}

// One thread per node of level l: P = mean of the four children's, then the fit.
__global__ void ggx_up(MapDesc d, int l, GgxDirs dirs, const float *__restrict__ Pc, float *__restrict__ Pp,
                       float4 *__restrict__ omega, uint32_t count)
{
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count) return;
    float Pl[kGgxDirs];
    bool ok = ggx_node_inside(d, l, m);
    for (int k = 0; k < kGgxDirs; ++k) {
        float v = 0.f;
        for (int c = 0; c < 4; ++c) v += Pc[(4 * size_t(m) + c) * kGgxDirs + k];
        Pl[k] = 0.25f * v;
        ok = ok && isfinite(Pl[k]);
    }
    for (int k = 0; k < kGgxDirs; ++k) Pp[size_t(m) * kGgxDirs + k] = ok ? Pl[k] : __int_as_float(0x7fc00000);
    float4 o = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
    if (ok && !ggx_fit(Pl, dirs, o)) o = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
    omega[m] = o;
}

GgxDirs make_ggx_dirs()
{
    GgxDirs g;
    const double r = sqrt(1.0 - double(kGgxWz) * kGgxWz);
    for (int k = 0; k < kGgxDirs; ++k) {
        const double ph = 2.0 * 3.14159265358979323846 * k / kGgxDirs;
        Dir &w = g.w[k];
        w.wx = float(r * cos(ph));
        w.wy = float(r * sin(ph));
        w.wz = kGgxWz;
        w.wr = sqrtf(w.wx * w.wx + w.wy * w.wy);
        w.c = w.wr > 0.f ? w.wx / w.wr : 1.f;
        w.s = w.wr > 0.f ? w.wy / w.wr : 0.f;
    }
    return g;
}

// Omega at a footprint: two mip levels around lambda = log2(sqrt(12) sigma),
// each bilinear between node centres, nodes without a fit dropped.
__device__ bool ggx_omega_at(const pndf_ggx &g, float x, float y, float sxx, float syy, float3 &O)
{
    const int L = g.L;
    float lam = log2f(3.4641016f * sqrtf(fmaxf(sxx, syy)));
    lam = fminf(fmaxf(lam, 2.0f), float(L));
    const int l0 = int(floorf(lam)), l1 = l0 < L ? l0 + 1 : l0;
    const float tl = lam - float(l0);
    float ax = 0.f, ay = 0.f, az = 0.f, wsum = 0.f;
    for (int side = 0; side < 2; ++side) {
        const int l = side ? l1 : l0;
        const float wl = side ? tl : 1.0f - tl;
        if (wl == 0.f) continue;
        const float a = float(1 << l);
        const int S = 1 << (L - l);
        const float fx = x / a - 0.5f, fy = y / a - 0.5f;
        const float flx = floorf(fx), fly = floorf(fy);
        const float tx = fx - flx, ty = fy - fly;
        float lx = 0.f, ly = 0.f, lz = 0.f, lw = 0.f;
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int I = int(fminf(fmaxf(flx + di, 0.f), float(S - 1)));
                const int J = int(fminf(fmaxf(fly + dj, 0.f), float(S - 1)));
                const float4 o = g.omega[l][morton2(uint32_t(I), uint32_t(J))];
                if (!isfinite(o.x)) continue;
                const float w = (di ? tx : 1.f - tx) * (dj ? ty : 1.f - ty);
                lx += w * o.x;
                ly += w * o.y;
                lz += w * o.z;
                lw += w;
            }
        if (lw > 0.f) {
            ax += wl * lx / lw;
            ay += wl * ly / lw;
            az += wl * lz / lw;
            wsum += wl;
        }
    }
    if (!(wsum > 0.f)) return false;
    O = make_float3(ax / wsum, ay / wsum, az / wsum);
    return true;
}

__device__ __forceinline__ float ggx_lambda(const float3 &O, float wx, float wy, float wz)
{
    const float qf = O.x * wx * wx + 2.0f * O.y * wx * wy + O.z * wy * wy;
    return 0.5f * (wz + sqrtf(fmaxf(wz * wz + qf, 0.f))) / wz - 1.0f;
}

__global__ void ggx_eval(pndf_ggx g, const pndf_query *__restrict__ q, const float *__restrict__ wi,
                         const float *__restrict__ wo, int64_t n, float *__restrict__ out)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const pndf_query r = q[k];
        float3 O;
        if (!(r.sxx > 0.f && r.syy > 0.f) || !ggx_omega_at(g, r.x, r.y, r.sxx, r.syy, O)) {
            out[k] = __int_as_float(0x7fc00000);
            continue;
        }
        const float ix = wi[3 * k], iy = wi[3 * k + 1], iz = wi[3 * k + 2];
        const float li = ggx_lambda(O, ix, iy, iz);
        if (!wo) {
            out[k] = li;
            continue;
        }
        // height-correlated shadow-masking with the query normal m
        const float ox = wo[3 * k], oy = wo[3 * k + 1], oz = wo[3 * k + 2];
        const float mz = sqrtf(fmaxf(0.f, 1.0f - r.ms * r.ms - r.mt * r.mt));
        const float ci = r.ms * ix + r.mt * iy + mz * iz, co = r.ms * ox + r.mt * oy + mz * oz;
        out[k] = (ci > 0.f && co > 0.f) ? 1.0f / (1.0f + li + ggx_lambda(O, ox, oy, oz)) : 0.f;
    }
}

__global__ void ggx_copy(pndf_ggx g, int l, float *__restrict__ out)
{
    const uint32_t S = 1u << (g.L - l);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * S) return;
    const float4 o = g.omega[l][morton2(i % S, i / S)];
    out[3 * size_t(i)] = o.x;
    out[3 * size_t(i) + 1] = o.y;
    out[3 * size_t(i) + 2] = o.z;
}

}  // namespace

pndf_status launch_ggx_build(const pndf_hierarchy *h, pndf_ggx *g, cudaStream_t s)
{
    const MapDesc &d = h->d;
    const int L = d.L;
    const uint32_t nleaf = uint32_t(level_nodes(L, kLeafLevel));
    const size_t pbytes = size_t(nleaf) * kGgxDirs * sizeof(float);
    void *scratch = nullptr;
    if (cudaMallocAsync(&scratch, 2 * pbytes, s) != cudaSuccess) {
        cudaGetLastError();
        return PNDF_ERR_OOM;
    }
    float *pa = static_cast<float *>(scratch), *pb = pa + size_t(nleaf) * kGgxDirs;
    static const GgxDirs dirs = make_ggx_dirs();
    const unsigned blocks = unsigned((size_t(nleaf) + kGgxLeafWarps - 1) / kGgxLeafWarps);
    if (d.texel_fmt == PNDF_TEXEL_F32X2)
        ggx_leaf<PNDF_TEXEL_F32X2><<<blocks, 32 * kGgxLeafWarps, 0, s>>>(d, dirs, pa, g->omega[kLeafLevel], nleaf);
    else
        ggx_leaf<PNDF_TEXEL_F16X2><<<blocks, 32 * kGgxLeafWarps, 0, s>>>(d, dirs, pa, g->omega[kLeafLevel], nleaf);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    for (int l = kLeafLevel + 1; e == cudaSuccess && l <= L; ++l) {
        const uint32_t cnt = uint32_t(level_nodes(L, l));
        ggx_up<<<(cnt + 127) / 128, 128, 0, s>>>(d, l, dirs, pa, pb, g->omega[l], cnt);
        count_launches(1);
        e = cudaGetLastError();
        float *t = pa;
        pa = pb;
        pb = t;
    }
    cudaError_t ef = cudaFreeAsync(scratch, s);
    return (e == cudaSuccess && ef == cudaSuccess) ? PNDF_OK : PNDF_ERR_CUDA;
}

cudaError_t launch_ggx_eval(const pndf_ggx *g, const pndf_query *q, const float *wi, const float *wo, int64_t n,
                            float *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + 255) / 256;
    if (blocks > int64_t(sms) * 16) blocks = int64_t(sms) * 16;
    ggx_eval<<<unsigned(blocks), 256, 0, s>>>(*g, q, wi, wo, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ggx_copy(const pndf_ggx *g, int l, float *out, cudaStream_t s)
{
    const uint32_t n = uint32_t(level_nodes(g->L, l));
    ggx_copy<<<(n + 255) / 256, 256, 0, s>>>(*g, l, out);
    count_launches(1);
    return cudaGetLastError();
}

int area_max_bands(int n) { return (n - 1 + kBand - 1) / kBand + 1; }

cudaError_t launch_area_step(int texel_fmt, const MapDesc *maps, int nmaps, const uint32_t *count,
                             const AreaReq *areq, int cap, uint32_t *off, float2 *part, unsigned int *cursor,
                             cudaStream_t s)
{
    if (cap <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    area_step_bands<<<(cap + 255) / 256, 256, 0, s>>>(maps, count, areq, off);
    area_step_scan<<<1, 1024, 0, s>>>(count, off);
    int occ = 0;
    if (texel_fmt == PNDF_TEXEL_F32X2) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, area_step_items<PNDF_TEXEL_F32X2>, 256, 0);
        area_step_items<PNDF_TEXEL_F32X2><<<sms * (occ > 0 ? occ : 1), 256, 0, s>>>(maps, nmaps, count, areq, off,
                                                                                    part, cursor);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, area_step_items<PNDF_TEXEL_F16X2>, 256, 0);
        area_step_items<PNDF_TEXEL_F16X2><<<sms * (occ > 0 ? occ : 1), 256, 0, s>>>(maps, nmaps, count, areq, off,
                                                                                    part, cursor);
    }
    area_step_reduce<<<(cap * 32 + 255) / 256, 256, 0, s>>>(maps, count, areq, off, part);
    return cudaGetLastError();
}

pndf_status launch_projarea(const pndf_hierarchy *h, const pndf_query *q, const float *omega, int64_t nq, float *P,
                            cudaStream_t s)
{
    if (nq == 0) return PNDF_OK;
    const MapDesc &d = h->d;
    const int maxbands = (d.n - 1 + kBand - 1) / kBand + 1;
    // requests per chunk: bounded by the scan (65536) and by 256 MiB of band partials
    int64_t chunk = (int64_t(1) << 28) / (int64_t(sizeof(float2)) * maxbands);
    if (chunk > 65536) chunk = 65536;
    if (chunk < 1024) chunk = 1024;
    if (chunk > nq) chunk = nq;
    size_t off_bytes = ((size_t(chunk) + 1) * sizeof(uint32_t) + 255) & ~size_t(255);
    size_t part_bytes = size_t(chunk) * maxbands * sizeof(float2);
    void *scratch = nullptr;
    if (cudaMallocAsync(&scratch, 256 + off_bytes + part_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return PNDF_ERR_OOM;
    }
    char *base = static_cast<char *>(scratch);
    auto *cursor = reinterpret_cast<unsigned int *>(base);
    auto *off = reinterpret_cast<uint32_t *>(base + 256);
    auto *part = reinterpret_cast<float2 *>(base + 256 + off_bytes);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    for (int64_t k0 = 0; k0 < nq && e == cudaSuccess; k0 += chunk) {
        int cnt = int(nq - k0 < chunk ? nq - k0 : chunk);
        e = cudaMemsetAsync(cursor, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) break;
        pa_bands<<<(cnt + 255) / 256, 256, 0, s>>>(d, q, k0, cnt, off);
        pa_scan<<<1, 1024, 0, s>>>(off, cnt);
        int occ = 0;
        if (d.texel_fmt == PNDF_TEXEL_F32X2) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pa_items<PNDF_TEXEL_F32X2>, 256, 0);
            pa_items<PNDF_TEXEL_F32X2><<<sms * (occ > 0 ? occ : 1), 256, 0, s>>>(d, q, omega, k0, cnt, off, part, cursor);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pa_items<PNDF_TEXEL_F16X2>, 256, 0);
            pa_items<PNDF_TEXEL_F16X2><<<sms * (occ > 0 ? occ : 1), 256, 0, s>>>(d, q, omega, k0, cnt, off, part, cursor);
        }
        pa_reduce<<<(cnt * 32 + 255) / 256, 256, 0, s>>>(q, k0, cnt, off, part, P, d.status);
        count_launches(4);
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess || ef != cudaSuccess) return PNDF_ERR_CUDA;
    return PNDF_OK;
}

namespace {
__global__ void take_projarea_word(unsigned int *out) { *out = atomicExch(&g_status_projarea, 0u); }
}  // namespace

cudaError_t take_status_projarea(unsigned int *out, cudaStream_t s)
{
    take_projarea_word<<<1, 1, 0, s>>>(out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pndf
