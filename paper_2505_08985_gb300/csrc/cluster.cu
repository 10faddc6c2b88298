// Cluster hierarchy build (Sec. 4.2 on mesh clustering, Eq. 7-8, App. A).
//
// Each node (level l >= 2, 2^l x 2^l quads, entirely inside the map) gets the
// four corner normals c00, c10, c01, c11 of a two-triangle cluster split like
// a quad (anti-diagonal) that minimise the Jacobian-weighted L2 error
//     F(c) = integral over the node of ||n^l(u) - n(u)||^2 / |det J(u)| du
// (Eq. 7), and the residual e = sqrt(F(c*)) of Eq. 8 (the 2-norm of the
// weighted error; units texel^2, like the r_x r_y of the cut criterion).  On
// a fine triangle |det J| is its |cross|, clamped below at 1e-6 like Eq. 6.
//
// F is a quadratic form in c.  On a fine triangle T (uv area 1/2, weight w =
// 1 / max(|cross|, 1e-6)) both n^l and n are linear, so with the cluster hats
// h(v) at T's vertices and d(v) = n^l(v) - n(v),
//     integral over T of w ||n^l - n||^2 = w / 24 (sum_v |d(v)|^2 + |sum_v d(v)|^2).
// A leaf block (4 x 4 quads) assembles G c = R from its 32 triangles, solves
// it, and sums F(c*) triangle by triangle: a sum of non-negative terms.
// Above the leaf level the parent's cluster restricted to a child lies in
// the child's own cluster space (linear on each child half; the parent's
// anti-diagonal runs along the children's), so with P_k the parent-corner to
// child-corner interpolation and the child's optimum (G_k, g_k, F_k),
//     F_parent(c) = sum_k F_k + (P_k c - g_k)^T G_k (P_k c - g_k),
// exact and again free of cancellation; the parent's normal equations are
// sum_k P_k^T G_k P_k c = sum_k P_k^T G_k g_k.  All of it is FP64.
//
// Kernel 1 (cluster_tiles): 256 threads per level-6 node (16 x 16 leaf
// blocks, Morton order): a thread fits one leaf block, levels 3 and 4 combine
// siblings by warp shuffles (every sibling lane adds its P_k terms and solves
// the parent's system), levels 5 and 6 through shared memory; level-6 forms
// go to a scratch array.  Kernel 2 (cluster_up): one launch per level above
// 6, one thread per node.
//
// The fitted corners can lie outside the hull of the texels they replace, so
// each node box is widened to hold its own cluster corners and its
// children's widened boxes: pruning by box never removes a cluster triangle
// that holds m, so the cut alone decides the result.
#include <math.h>

#include "common.cuh"

namespace pndf {
namespace {

constexpr double kJacEps = 1e-6;

// A node's quadratic form at its optimum: Gram matrix G (symmetric, upper
// triangle packed: 00 01 02 03 11 12 13 22 23 33), optimal corners g
// (c00, c10, c01, c11 as (s, t)) and minimum F.
struct QF {
    double G[10];
    double g[4][2];
    double F;
};

__host__ __device__ constexpr int sym_ordered(int a, int b) { return a * 4 - a * (a - 1) / 2 + (b - a); }
__host__ __device__ constexpr int sym(int a, int b) { return a <= b ? sym_ordered(a, b) : sym_ordered(b, a); }

// Cluster hats at normalised local (s, t): lower half (s + t <= 1) 1 - s - t,
// s, t, 0; upper half 0, 1 - t, 1 - s, s + t - 1 (both agree on the diagonal).
__host__ __device__ constexpr double hat(int a, double s, double t)
{
    return s + t <= 1.0 ? (a == 0 ? 1.0 - s - t : a == 1 ? s : a == 2 ? t : 0.0)
                        : (a == 0 ? 0.0 : a == 1 ? 1.0 - t : a == 2 ? 1.0 - s : s + t - 1.0);
}

// Cholesky solve of G c = R (G packed symmetric).  False if G is not
// numerically positive definite.
__host__ __device__ bool solve_spd(const double Gp[10], const double R[4][2], double c[4][2])
{
    double L[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double d = Gp[sym(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        L[j][j] = d;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            double v = Gp[sym(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v / d;
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        double y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            double v = R[i][r];
#pragma unroll
            for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
            y[i] = v / L[i][i];
        }
#pragma unroll
        for (int i = 3; i >= 0; --i) {
            double v = y[i];
#pragma unroll
            for (int k = i + 1; k < 4; ++k) v -= L[k][i] * c[k][r];
            c[i][r] = v / L[i][i];
        }
    }
    return true;
}

// A fine triangle of a leaf block: local texel coordinates of its vertices
// (tri 0: (qi, qj), (qi+1, qj), (qi, qj+1); tri 1: (qi+1, qj+1), (qi, qj+1),
// (qi+1, qj)) and the cluster half holding it (centroid s + t < 1).
__host__ __device__ constexpr int vx(int qi, int tri, int v) { return tri ? (v == 1 ? qi : qi + 1) : (v == 1 ? qi + 1 : qi); }
__host__ __device__ constexpr int vy(int qj, int tri, int v) { return tri ? (v == 2 ? qj : qj + 1) : (v == 2 ? qj + 1 : qj); }

template <int TFMT>
__device__ __forceinline__ float2 texel_at(const MapDesc &d, int i, int j)
{
    size_t idx = size_t(j) * d.n + i;
    if (TFMT == PNDF_TEXEL_F32X2) return __ldg(reinterpret_cast<const float2 *>(d.texels) + idx);
    return __half22float2(__ldg(reinterpret_cast<const __half2 *>(d.texels) + idx));
}

// Fit of leaf block (I, J) (4 x 4 quads), all of whose quads lie in the map.
// Returns false if the normal equations are singular.
// Fit of a leaf block (4 x 4 quads) from its 5 x 5 texels tx[y][x].
// Returns false if the normal equations are singular.
__host__ __device__ bool leaf_fit_texels(const float2 (&tx)[kLeafQuads + 1][kLeafQuads + 1], QF &out)
{
    constexpr int Q = kLeafQuads;
    double G[10], R[4][2];
#pragma unroll
    for (int k = 0; k < 10; ++k) G[k] = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) R[a][0] = R[a][1] = 0.0;
    // pass 1: normal equations
#pragma unroll
    for (int qj = 0; qj < Q; ++qj)
#pragma unroll
        for (int qi = 0; qi < Q; ++qi)
#pragma unroll
            for (int tri = 0; tri < 2; ++tri) {
                // cluster half by the centroid: lower iff qi + qj <= Q - 1 (tri 0), Q - 2 (tri 1)
                const int base = qi + qj <= Q - 1 - tri ? 0 : 1;  // active hats base..base+2
                double nx[3], ny[3], h[3][3];
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int x = vx(qi, tri, v), y = vy(qj, tri, v);
                    nx[v] = tx[y][x].x;
                    ny[v] = tx[y][x].y;
#pragma unroll
                    for (int k = 0; k < 3; ++k) h[v][k] = hat(base + k, double(x) / Q, double(y) / Q);
                }
                const double cr = (nx[1] - nx[0]) * (ny[2] - ny[0]) - (ny[1] - ny[0]) * (nx[2] - nx[0]);
                const double w = (1.0 / 24.0) / fmax(fabs(cr), kJacEps);
                const double sx = nx[0] + nx[1] + nx[2], sy = ny[0] + ny[1] + ny[2];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double hk = h[0][k] + h[1][k] + h[2][k];
                    R[base + k][0] += w * (h[0][k] * nx[0] + h[1][k] * nx[1] + h[2][k] * nx[2] + hk * sx);
                    R[base + k][1] += w * (h[0][k] * ny[0] + h[1][k] * ny[1] + h[2][k] * ny[2] + hk * sy);
#pragma unroll
                    for (int k2 = k; k2 < 3; ++k2) {
                        const double hk2 = h[0][k2] + h[1][k2] + h[2][k2];
                        G[sym(base + k, base + k2)] +=
                            w * (h[0][k] * h[0][k2] + h[1][k] * h[1][k2] + h[2][k] * h[2][k2] + hk * hk2);
                    }
                }
            }
    if (!solve_spd(G, R, out.g)) return false;
    // pass 2: F(c*) as a sum of non-negative terms
    double F = 0.0;
#pragma unroll
    for (int qj = 0; qj < Q; ++qj)
#pragma unroll
        for (int qi = 0; qi < Q; ++qi)
#pragma unroll
            for (int tri = 0; tri < 2; ++tri) {
                const int base = qi + qj <= Q - 1 - tri ? 0 : 1;
                double nx[3], ny[3], dx[3], dy[3];
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int x = vx(qi, tri, v), y = vy(qj, tri, v);
                    nx[v] = tx[y][x].x;
                    ny[v] = tx[y][x].y;
                    double ax = 0.0, ay = 0.0;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const double hv = hat(base + k, double(x) / Q, double(y) / Q);
                        ax += hv * out.g[base + k][0];
                        ay += hv * out.g[base + k][1];
                    }
                    dx[v] = ax - nx[v];
                    dy[v] = ay - ny[v];
                }
                const double cr = (nx[1] - nx[0]) * (ny[2] - ny[0]) - (ny[1] - ny[0]) * (nx[2] - nx[0]);
                const double w = (1.0 / 24.0) / fmax(fabs(cr), kJacEps);
                const double sx = dx[0] + dx[1] + dx[2], sy = dy[0] + dy[1] + dy[2];
                F += w * (dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2] + dy[0] * dy[0] + dy[1] * dy[1] +
                          dy[2] * dy[2] + sx * sx + sy * sy);
            }
#pragma unroll
    for (int k = 0; k < 10; ++k) out.G[k] = G[k];
    out.F = F;
    return true;
}

// Fit of leaf block (I, J), all of whose quads lie in the map.
template <int TFMT>
__device__ bool leaf_fit(const MapDesc &d, uint32_t I, uint32_t J, QF &out)
{
    constexpr int Q = kLeafQuads;
    const int i0 = int(I) * Q, j0 = int(J) * Q;
    float2 tx[Q + 1][Q + 1];
#pragma unroll
    for (int y = 0; y <= Q; ++y)
#pragma unroll
        for (int x = 0; x <= Q; ++x) tx[y][x] = texel_at<TFMT>(d, i0 + x, j0 + y);
    return leaf_fit_texels(tx, out);
}

// Child (ox, oy) of a parent: P[j][a] = parent hat a at child corner j, in
// the parent's frame.
__host__ __device__ __forceinline__ void child_interp(int ox, int oy, double P[4][4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int a = 0; a < 4; ++a) P[j][a] = hat(a, 0.5 * (ox + (j & 1)), 0.5 * (oy + (j >> 1)));
}

// The child's terms of its parent's normal equations: P^T G P (packed) and P^T G g.
__host__ __device__ __forceinline__ void child_terms(const QF &c, int ox, int oy, double CG[10], double CR[4][2])
{
    double P[4][4], GP[4][4];
    child_interp(ox, oy, P);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < 4; ++j) v += c.G[sym(i, j)] * P[j][a];
            GP[i][a] = v;
        }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
            double v = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) v += P[i][a] * GP[i][b];
            CG[sym(a, b)] = v;
        }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            double v = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) v += GP[i][a] * c.g[i][r];
            CR[a][r] = v;
        }
}

// The child's share of F_parent(cp): F_k + (P cp - g)^T G (P cp - g).
__host__ __device__ __forceinline__ double child_misfit(const QF &c, int ox, int oy, const double cp[4][2])
{
    double P[4][4];
    child_interp(ox, oy, P);
    double F = c.F;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        double D[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double v = -c.g[j][r];
#pragma unroll
            for (int a = 0; a < 4; ++a) v += P[j][a] * cp[a][r];
            D[j] = v;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < 4; ++j) v += c.G[sym(i, j)] * D[j];
            F += D[i] * v;
        }
    }
    return F;
}

// Parent of four children held in memory (Morton order k = dy * 2 + dx).
__host__ __device__ bool combine4(const QF ch[4], QF &out)
{
    double G[10], R[4][2];
#pragma unroll
    for (int k = 0; k < 10; ++k) G[k] = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) R[a][0] = R[a][1] = 0.0;
    for (int k = 0; k < 4; ++k) {
        double CG[10], CR[4][2];
        child_terms(ch[k], k & 1, k >> 1, CG, CR);
#pragma unroll
        for (int t = 0; t < 10; ++t) G[t] += CG[t];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            R[a][0] += CR[a][0];
            R[a][1] += CR[a][1];
        }
    }
    if (!solve_spd(G, R, out.g)) return false;
    double F = 0.0;
    for (int k = 0; k < 4; ++k) F += child_misfit(ch[k], k & 1, k >> 1, out.g);
#pragma unroll
    for (int t = 0; t < 10; ++t) out.G[t] = G[t];
    out.F = F;
    return true;
}

// Parent of the four sibling lanes (lane bits sh, sh + 1 give the child
// offset): every sibling ends with the parent's form.
__device__ bool combine_lanes(QF &m, int ox, int oy, int sh)
{
    double G[10], R[4][2];
    child_terms(m, ox, oy, G, R);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int mask = 1 << (sh + b);
#pragma unroll
        for (int t = 0; t < 10; ++t) G[t] += __shfl_xor_sync(0xffffffffu, G[t], mask);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            R[a][0] += __shfl_xor_sync(0xffffffffu, R[a][0], mask);
            R[a][1] += __shfl_xor_sync(0xffffffffu, R[a][1], mask);
        }
    }
    double cp[4][2];
    const bool ok = solve_spd(G, R, cp);
    double F = ok ? child_misfit(m, ox, oy, cp) : 0.0;
#pragma unroll
    for (int b = 0; b < 2; ++b) F += __shfl_xor_sync(0xffffffffu, F, 1 << (sh + b));
#pragma unroll
    for (int t = 0; t < 10; ++t) m.G[t] = G[t];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        m.g[a][0] = cp[a][0];
        m.g[a][1] = cp[a][1];
    }
    m.F = F;
    return ok;
}

__device__ __forceinline__ void widen_corner(Box &b, float c0, float c1, float d0, float d1)
{
    b.smin = fminf(b.smin, __fadd_rd(c0, d0));
    b.tmin = fminf(b.tmin, __fadd_rd(c1, d1));
    b.smax = fmaxf(b.smax, __fadd_ru(c0, d0));
    b.tmax = fmaxf(b.tmax, __fadd_ru(c1, d1));
}

// Store node m of level l (fitted, with form qf, when ok) and widen its box
// (own corners + children's widened boxes, which this launch or the previous
// one has already written).
template <int BFMT>
__device__ void fit_store(const MapDesc &d, const ClusterDesc &cd, int l, uint32_t m, bool ok, const QF &qf)
{
    const uint32_t I = compact1by1(m), J = compact1by1(m >> 1);
    const int64_t a = int64_t(1) << l;
    ok = ok && a * (I + 1) <= int64_t(d.n) - 1 && a * (J + 1) <= int64_t(d.n) - 1;
    float4 *rec = const_cast<float4 *>(cd.cl[l]) + 2 * size_t(m);
    float *ev = const_cast<float *>(cd.ce[l]) + m;
    Box b = load_box<BFMT>(d.lv[l], m);
    if (l > kLeafLevel) {
#pragma unroll
        for (int k = 0; k < 4; ++k) grow(b, load_box<BFMT>(d.lv[l - 1], 4 * size_t(m) + k));
    }
    if (ok) {
        const double(*c)[2] = qf.g;
        float c0 = float(c[0][0]), c1 = float(c[0][1]);
        float d10x = float(c[1][0] - c[0][0]), d10y = float(c[1][1] - c[0][1]);
        float d01x = float(c[2][0] - c[0][0]), d01y = float(c[2][1] - c[0][1]);
        float d11x = float(c[3][0] - c[0][0]), d11y = float(c[3][1] - c[0][1]);
        rec[0] = make_float4(c0, c1, d10x, d10y);
        rec[1] = make_float4(d01x, d01y, d11x, d11y);
        *ev = float(sqrt(fmax(qf.F, 0.0)));
        widen_corner(b, c0, c1, 0.f, 0.f);
        widen_corner(b, c0, c1, d10x, d10y);
        widen_corner(b, c0, c1, d01x, d01y);
        widen_corner(b, c0, c1, d11x, d11y);
    } else {
        rec[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        *ev = __int_as_float(0x7f800000);
    }
    store_box<BFMT>(const_cast<void *>(d.lv[l]), m, b);
}

// A node's fit is valid only if all its quads lie in the map (then so do its
// children's) and every solve on the way succeeded.
__device__ __forceinline__ bool node_inside_map(const MapDesc &d, int l, uint32_t m)
{
    const int64_t a = int64_t(1) << l;
    return a * (compact1by1(m) + 1) <= int64_t(d.n) - 1 && a * (compact1by1(m >> 1) + 1) <= int64_t(d.n) - 1;
}

constexpr int kTileLevels = 4;                        // levels 3..6 above the leaf level in one CTA
constexpr int kTileThreads = 1 << (2 * kTileLevels);  // 256 leaf blocks

// Two CTAs per SM (128 registers, the rest spilled): 32.1 ms against 38.3 ms
// at one (255 registers) for the 8192^2 cluster hierarchy; the FP64 pipe
// needs the second CTA's warps to stay busy.
template <int TFMT, int BFMT>
__global__ void __launch_bounds__(kTileThreads, 2) cluster_tiles(MapDesc d, ClusterDesc cd, QF *__restrict__ out6)
{
    __shared__ QF part[16];
    __shared__ bool part_ok[16];
    const int tid = threadIdx.x;
    const int L = d.L;
    const uint32_t m2 = blockIdx.x * kTileThreads + tid;  // leaf block, Morton order
    const uint32_t n2 = uint32_t(level_nodes(L, kLeafLevel));
    QF m;
    bool ok = false;
    if (m2 < n2) {
        ok = node_inside_map(d, kLeafLevel, m2) && leaf_fit<TFMT>(d, compact1by1(m2), compact1by1(m2 >> 1), m);
        fit_store<BFMT>(d, cd, kLeafLevel, m2, ok, m);
    }
    if (!ok) {  // keep the shuffled sums finite; such a node's ancestors are never fitted
#pragma unroll
        for (int t = 0; t < 10; ++t) m.G[t] = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) m.g[a][0] = m.g[a][1] = 0.0;
        m.F = 0.0;
    }
    // levels 3 and 4: siblings are 4 lanes apart by 1, 2 (level 3) or 4, 8 (level 4)
#pragma unroll
    for (int k = 1; k <= 2; ++k) {
        const int l = kLeafLevel + k, sh = 2 * (k - 1);
        // every lane takes part in every shuffle (no short-circuit around them)
        int sib_ok = ok ? 1 : 0;
        sib_ok &= __shfl_xor_sync(0xffffffffu, sib_ok, 1 << sh);
        sib_ok &= __shfl_xor_sync(0xffffffffu, sib_ok, 2 << sh);
        const bool fit_ok = combine_lanes(m, (tid >> sh) & 1, (tid >> (sh + 1)) & 1, sh);
        ok = fit_ok && sib_ok != 0;
        __syncthreads();  // children's boxes are written
        const uint32_t ml = m2 >> (2 * k);
        if (l <= L && (tid & ((1 << (2 * k)) - 1)) == 0 && ml < uint32_t(level_nodes(L, l)))
            fit_store<BFMT>(d, cd, l, ml, ok && node_inside_map(d, l, ml), m);
    }
    // level 5 from the 16 level-4 nodes of the block, level 6 from the four level-5 nodes
    if ((tid & 15) == 0) {
        part[tid >> 4] = m;
        part_ok[tid >> 4] = ok;
    }
    __syncthreads();
    QF p5;
    bool ok5 = false;
    if (tid < 4) {
        ok5 = part_ok[4 * tid] && part_ok[4 * tid + 1] && part_ok[4 * tid + 2] && part_ok[4 * tid + 3] &&
              combine4(&part[4 * tid], p5);
        const uint32_t ml = (blockIdx.x << 2) | uint32_t(tid);
        if (kLeafLevel + 3 <= L && ml < uint32_t(level_nodes(L, kLeafLevel + 3)))
            fit_store<BFMT>(d, cd, kLeafLevel + 3, ml, ok5 && node_inside_map(d, kLeafLevel + 3, ml), p5);
    }
    __syncthreads();
    if (tid < 4) {
        part[tid] = p5;
        part_ok[tid] = ok5;
    }
    __syncthreads();
    if (tid == 0 && kLeafLevel + 4 <= L) {
        QF p6;
        bool ok6 = part_ok[0] && part_ok[1] && part_ok[2] && part_ok[3] && combine4(part, p6);
        fit_store<BFMT>(d, cd, kLeafLevel + 4, blockIdx.x, ok6 && node_inside_map(d, kLeafLevel + 4, blockIdx.x),
                        p6);
        if (out6) {
            if (!ok6) p6.F = -1.0;  // marks an invalid form for the level above
            out6[blockIdx.x] = p6;
        }
    }
}

template <int BFMT>
__global__ void cluster_up(MapDesc d, ClusterDesc cd, int l, const QF *__restrict__ in, QF *__restrict__ out,
                           uint32_t count)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    QF ch[4];
    bool ok = node_inside_map(d, l, i);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ch[k] = in[4 * size_t(i) + k];
        ok = ok && ch[k].F >= 0.0;
    }
    QF p;
    ok = ok && combine4(ch, p);
    fit_store<BFMT>(d, cd, l, i, ok, p);
    if (out) {
        if (!ok) p.F = -1.0;
        out[i] = p;
    }
}

template <int TFMT, int BFMT>
cudaError_t launch_clusters_t(pndf_hierarchy *h, cudaStream_t s)
{
    const MapDesc &d = h->d;
    const int L = d.L;
    const int top_tile = kLeafLevel + kTileLevels;  // 6
    const unsigned blocks = L >= top_tile ? unsigned(level_nodes(L, top_tile)) : 1u;
    QF *a = static_cast<QF *>(h->moments);
    QF *b = a ? a + level_nodes(L, top_tile) : nullptr;
    cluster_tiles<TFMT, BFMT><<<blocks, kTileThreads, 0, s>>>(d, h->c, L > top_tile ? a : nullptr);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    for (int l = top_tile + 1; e == cudaSuccess && l <= L; ++l) {
        const uint32_t cnt = uint32_t(level_nodes(L, l));
        cluster_up<BFMT><<<(cnt + 127) / 128, 128, 0, s>>>(d, h->c, l, a, l < L ? b : nullptr, cnt);
        count_launches(1);
        e = cudaGetLastError();
        QF *t = a;
        a = b;
        b = t;
    }
    return e;
}

// Copy level l's records and residuals out in row-major node order (J, I).
__global__ void cluster_copy(ClusterDesc cd, int L, int l, float *__restrict__ rec, float *__restrict__ e)
{
    const uint32_t S = 1u << (L - l);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * S) return;
    const uint32_t m = morton2(i % S, i / S);
    float4 r0 = cd.cl[l][2 * size_t(m)], r1 = cd.cl[l][2 * size_t(m) + 1];
    float *o = rec + 8 * size_t(i);
    o[0] = r0.x; o[1] = r0.y; o[2] = r0.z; o[3] = r0.w;
    o[4] = r1.x; o[5] = r1.y; o[6] = r1.z; o[7] = r1.w;
    e[i] = cd.ce[l][m];
}

}  // namespace

cudaError_t launch_cluster_copy(const pndf_hierarchy *h, int l, float *rec, float *e, cudaStream_t s)
{
    const uint32_t n = uint32_t(level_nodes(h->d.L, l));
    cluster_copy<<<(n + 255) / 256, 256, 0, s>>>(h->c, h->d.L, l, rec, e);
    count_launches(1);
    return cudaGetLastError();
}

size_t cluster_scratch_bytes(int L)
{
    const int top_tile = kLeafLevel + kTileLevels;
    if (L <= top_tile) return 0;
    return (level_nodes(L, top_tile) + level_nodes(L, top_tile + 1)) * sizeof(QF);
}

cudaError_t launch_clusters(pndf_hierarchy *h, cudaStream_t s)
{
    const MapDesc &d = h->d;
    if (d.texel_fmt == PNDF_TEXEL_F32X2)
        return d.bounds_fmt == PNDF_BOUNDS_F32 ? launch_clusters_t<PNDF_TEXEL_F32X2, PNDF_BOUNDS_F32>(h, s)
                                               : launch_clusters_t<PNDF_TEXEL_F32X2, PNDF_BOUNDS_F16_OUTWARD>(h, s);
    return d.bounds_fmt == PNDF_BOUNDS_F32 ? launch_clusters_t<PNDF_TEXEL_F16X2, PNDF_BOUNDS_F32>(h, s)
                                           : launch_clusters_t<PNDF_TEXEL_F16X2, PNDF_BOUNDS_F16_OUTWARD>(h, s);
}

}  // namespace pndf
