/*
 * FP64 CPU oracle for the position-normal-manifold P-NDF and the analytic
 * projected-area integral.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA path.  It is a plain,
 * slow, exhaustive evaluation: no hierarchy, no blocking, no reordering.
 *
 * Map layout: st[(j*N + i)*2 + c], texel u = (i, j), c = 0 for s, 1 for t.
 * Query layout: 7 doubles (x, y, sxx, sxy, syy, ms, mt).
 * Triangulation (Eq. 3, Tab. 1): quad (i, j), 0 <= i, j <= N-2, with corners
 *   u0 = (i, j), u1 = (i+1, j), u2 = (i, j+1), u3 = (i+1, j+1);
 *   lower triangle (u0, u1, u2) where u+v < 1, upper triangle (u3, u2, u1).
 * Triangle id = 2 * (j*(N-1) + i) + (0 lower | 1 upper).
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *  - Footprint kernel: Gaussian exp(-q/2) / (2 pi sqrt(det Sigma)) with
 *    q = d^T Sigma^-1 d, cut to zero where q > 16 (the 4-sigma ellipse);
 *    not renormalised.
 *  - Domain: non-periodic; only quads inside the map exist.
 *  - Hit indicator (Eq. 5): all three barycentrics >= 0 (closed).  A
 *    triangle with exactly zero normal-space area is a delta, not a density,
 *    and is skipped.
 *  - Projected area, k_r(T): the Gaussian at the uv centroid of T, with the
 *    same 16 cut at the centroid.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define ORACLE_QCUT 16.0
#define ORACLE_EDGE_EPS 1e-6
#define ORACLE_CUT_EPS 1e-4
#define ORACLE_TINY_AREA 1e-10

enum {
    OF_NEAR_EDGE = 1u,   /* m within 1e-6 of an edge of a footprint triangle     */
    OF_NEAR_CUT = 2u,    /* a hit with |q - 16| <= 1e-4                           */
    OF_DEGENERATE = 4u,  /* m within 1e-6 of a zero-area normal triangle          */
    OF_TINY = 8u,        /* a hit on a triangle of normal-space area < 1e-10      */
    OF_INVALID = 16u     /* covariance not positive definite                      */
};

/* MurmurHash3 32-bit finalizer (Appleby), used only to fingerprint hit sets. */
static uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* Twice the signed area of triangle (p, q, r): (q - p) x (r - p). */
static double area2(double px, double py, double qx, double qy, double rx, double ry)
{
    return (qx - px) * (ry - py) - (qy - py) * (rx - px);
}

/* Distance from point m to segment [a, b]. */
static double seg_dist(double mx, double my, double ax, double ay, double bx, double by)
{
    double vx = bx - ax, vy = by - ay;
    double wx = mx - ax, wy = my - ay;
    double L2 = vx * vx + vy * vy;
    double t = L2 > 0.0 ? (wx * vx + wy * vy) / L2 : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double dx = wx - t * vx, dy = wy - t * vy;
    return sqrt(dx * dx + dy * dy);
}

static void texel(const double *st, int N, int i, int j, double n[2])
{
    n[0] = st[((size_t)j * N + i) * 2 + 0];
    n[1] = st[((size_t)j * N + i) * 2 + 1];
}

/* Quads whose uv square [i, i+1] x [j, j+1] can meet the bounding box of the
 * 4-sigma ellipse; a generous superset is harmless (Eq. 5: triangles outside
 * the footprint contribute k_r = 0). */
static void quad_range(int N, double x, double y, double sxx, double syy,
                       int *i0, int *i1, int *j0, int *j1)
{
    double rx = 4.0 * sqrt(sxx), ry = 4.0 * sqrt(syy);
    double a = floor(x - rx) - 1.0, b = ceil(x + rx) + 1.0;
    double c = floor(y - ry) - 1.0, d = ceil(y + ry) + 1.0;
    if (a < 0) a = 0;
    if (c < 0) c = 0;
    if (b > N - 2) b = N - 2;
    if (d > N - 2) d = N - 2;
    *i0 = (int)a; *i1 = (int)b; *j0 = (int)c; *j1 = (int)d;
}

/*
 * P-NDF of one query by exhaustive summation, Eq. 5 (the closed-form
 * solution of Eq. 2): D(m, x) = sum over triangles abc with m in n(abc) of
 * k_r(a l0 + b l1 + c l2 - x) / (2 ||n(abc)||), where (l0, l1, l2) =
 * bary(m, n(abc)) from signed areas (Tab. 1) and 2 ||n(abc)|| is the
 * Jacobian of Eq. 4, i.e. |(n_b - n_a) x (n_c - n_a)|.
 */
static void pndf_one(const double *st, int N, const double *qq,
                     double *D_out, uint32_t *flags_out, int64_t *nhits_out, uint32_t *hash_out)
{
    double x = qq[0], y = qq[1], sxx = qq[2], sxy = qq[3], syy = qq[4], mx = qq[5], my = qq[6];
    double det = sxx * syy - sxy * sxy;
    uint32_t flags = 0;
    if (!(sxx > 0.0) || !(syy > 0.0) || !(det > 0.0)) {
        *D_out = NAN;
        *flags_out = OF_INVALID;
        *nhits_out = 0;
        *hash_out = 0;
        return;
    }
    /* Sigma^-1 = [syy, -sxy; -sxy, sxx] / det */
    double ia = syy / det, ib = -sxy / det, ic = sxx / det;
    double norm = 1.0 / (2.0 * M_PI * sqrt(det));
    int i0, i1, j0, j1;
    quad_range(N, x, y, sxx, syy, &i0, &i1, &j0, &j1);
    double D = 0.0;
    int64_t nh = 0;
    uint32_t hsum = 0;
    for (int j = j0; j <= j1; ++j) {
        for (int i = i0; i <= i1; ++i) {
            double n0[2], n1[2], n2[2], n3[2];
            texel(st, N, i, j, n0);
            texel(st, N, i + 1, j, n1);
            texel(st, N, i, j + 1, n2);
            texel(st, N, i + 1, j + 1, n3);
            for (int tri = 0; tri < 2; ++tri) {
                /* uv vertices a, b, c and their normals */
                double ax, ay, bx, by, cx, cy;
                const double *na, *nb, *nc;
                if (tri == 0) {           /* (u0, u1, u2) */
                    ax = i; ay = j; bx = i + 1; by = j; cx = i; cy = j + 1;
                    na = n0; nb = n1; nc = n2;
                } else {                  /* (u3, u2, u1) */
                    ax = i + 1; ay = j + 1; bx = i; by = j + 1; cx = i + 1; cy = j;
                    na = n3; nb = n2; nc = n1;
                }
                double A2 = area2(na[0], na[1], nb[0], nb[1], nc[0], nc[1]);
                /* edge proximity census (footprint triangles only) */
                double lox = fmin(na[0], fmin(nb[0], nc[0])) - ORACLE_EDGE_EPS;
                double hix = fmax(na[0], fmax(nb[0], nc[0])) + ORACLE_EDGE_EPS;
                double loy = fmin(na[1], fmin(nb[1], nc[1])) - ORACLE_EDGE_EPS;
                double hiy = fmax(na[1], fmax(nb[1], nc[1])) + ORACLE_EDGE_EPS;
                if (mx >= lox && mx <= hix && my >= loy && my <= hiy) {
                    double dmin = seg_dist(mx, my, na[0], na[1], nb[0], nb[1]);
                    dmin = fmin(dmin, seg_dist(mx, my, nb[0], nb[1], nc[0], nc[1]));
                    dmin = fmin(dmin, seg_dist(mx, my, nc[0], nc[1], na[0], na[1]));
                    if (dmin <= ORACLE_EDGE_EPS) flags |= (A2 == 0.0) ? (OF_NEAR_EDGE | OF_DEGENERATE) : OF_NEAR_EDGE;
                }
                if (A2 == 0.0) continue;
                /* bary(m, n(abc)) = (|m b c|, |a m c|, |a b m|) / |a b c| (Tab. 1) */
                double l0 = area2(mx, my, nb[0], nb[1], nc[0], nc[1]) / A2;
                double l1 = area2(na[0], na[1], mx, my, nc[0], nc[1]) / A2;
                double l2 = area2(na[0], na[1], nb[0], nb[1], mx, my) / A2;
                if (!(l0 >= 0.0 && l1 >= 0.0 && l2 >= 0.0)) continue;
                /* the intersection's uv coordinate, then the footprint kernel */
                double ux = ax * l0 + bx * l1 + cx * l2;
                double uy = ay * l0 + by * l1 + cy * l2;
                double dx = ux - x, dy = uy - y;
                double q = ia * dx * dx + 2.0 * ib * dx * dy + ic * dy * dy;
                if (fabs(q - ORACLE_QCUT) <= ORACLE_CUT_EPS) flags |= OF_NEAR_CUT;
                if (q > ORACLE_QCUT) continue;
                double J = fabs(A2);
                if (0.5 * J < ORACLE_TINY_AREA) flags |= OF_TINY;
                D += norm * exp(-0.5 * q) / J;
                nh += 1;
                uint32_t id = (uint32_t)(2u * ((uint32_t)j * (uint32_t)(N - 1) + (uint32_t)i) + (uint32_t)tri);
                hsum += fmix32(id);
            }
        }
    }
    *D_out = D;
    *flags_out = flags;
    *nhits_out = nh;
    *hash_out = hsum;
}

/* Evaluate queries [k0, k1).  Safe to call concurrently on disjoint ranges. */
void oracle_pndf(const double *st, int N, const double *q, int64_t k0, int64_t k1,
                 double *D, uint32_t *flags, int64_t *nhits, uint32_t *hsum)
{
    for (int64_t k = k0; k < k1; ++k)
        pndf_one(st, N, q + 7 * k, D + k, flags + k, nhits + k, hsum + k);
}

/* ------------------------------------------------------------------------- */
/* Projected area, Eq. 9-11 and Alg. 1 (App. B).                             */
/* ------------------------------------------------------------------------- */

/* 2 * integral of sqrt(1 - p^2): F(p) = asin p + p sqrt(1 - p^2). */
static double Fasin(double p)
{
    if (p > 1.0) p = 1.0;
    if (p < -1.0) p = -1.0;
    return asin(p) + p * sqrt(1.0 - p * p);
}

/*
 * Alg. 1 (clip triangle edge) in the rotated frame (omega_y = 0, omega_x >= 0).
 * The invisible part of the projected disk is {m_x < 0, (m_x / w_z)^2 + m_y^2 > 1}.
 * Returns 0 when the edge is dropped, else the clipped endpoints and whether
 * each end was moved onto the ellipse.
 */
static int clip_edge(const double a[2], const double b[2], double wz,
                     double oa[2], double ob[2], int *ca, int *cb)
{
    double dx = b[0] - a[0], dy = b[1] - a[1];
    double w2 = wz * wz;
    double A = w2 * dy * dy + dx * dx;
    double B = 2.0 * (w2 * a[1] * dy + a[0] * dx);
    double C = w2 * (a[1] * a[1] - 1.0) + a[0] * a[0];
    double C1 = w2 * (b[1] * b[1] - 1.0) + b[0] * b[0];
    double disc = B * B - 4.0 * A * C;
    int clip0 = (C > 0.0) && (a[0] < 0.0);
    int clip1 = (C1 > 0.0) && (b[0] < 0.0);
    oa[0] = a[0]; oa[1] = a[1];
    ob[0] = b[0]; ob[1] = b[1];
    *ca = 0; *cb = 0;
    if (clip0 || clip1) {
        if (disc < 0.0) return 0;
        double sq = sqrt(disc);
        double t0 = (-B - sq) / (2.0 * A);
        double t1 = (-B + sq) / (2.0 * A);
        if (clip0) {
            oa[0] = a[0] * (1.0 - t0) + b[0] * t0;
            oa[1] = a[1] * (1.0 - t0) + b[1] * t0;
            *ca = 1;
        }
        if (clip1) {
            ob[0] = a[0] * (1.0 - t1) + b[0] * t1;
            ob[1] = a[1] * (1.0 - t1) + b[1] * t1;
            *cb = 1;
        }
        if (clip0 && clip1 && (t0 < 0.0 || t0 > 1.0 || t1 < 0.0 || t1 > 1.0)) return 0;
    }
    return 1;
}

/*
 * Eq. 11, line segment p -> q: the boundary integral of
 * (w_z m_x - w_x m~_z) dm_y.  The w_z part is (w_z/2)(q_y - p_y)(q_x + p_x).
 * The w_x part integrates m~_z = sqrt(r^2 - s^2) along the line, where the
 * line's distance to the origin is |d_y p_x - d_x p_y| and r^2 = 1 - that^2
 * (App. B, "line segments"); it enters with a minus sign because the
 * integrand is w_z m~_x - w_x m~_z.  dm_y = d_y dp (the printed "d_x" for the
 * projection cosine does not match the formula beside it, which uses d_y).
 */
static double line_term(const double p[2], const double q[2], double wx, double wz)
{
    double tz = 0.5 * wz * (q[1] - p[1]) * (q[0] + p[0]);
    double ex = q[0] - p[0], ey = q[1] - p[1];
    double len = sqrt(ex * ex + ey * ey);
    if (len == 0.0) return 0.0;
    double dx = ex / len, dy = ey / len;
    double s = dy * p[0] - dx * p[1];
    double r2 = 1.0 - s * s;
    double r = sqrt(r2);
    double pp = (dx * p[0] + dy * p[1]) / r;
    double pq = (dx * q[0] + dy * q[1]) / r;
    double tx = 0.5 * wx * r2 * dy * (Fasin(pq) - Fasin(pp));
    return tz - tx;
}

/* Eq. 11, ellipse arc from e to s: (1/2) [F(e_y) - F(s_y)]. */
static double arc_term(const double e[2], const double s[2])
{
    return 0.5 * (Fasin(e[1]) - Fasin(s[1]));
}

/*
 * Integral over n+(T) = n(T) intersected with the visible region of
 * (w_x m~_x / m~_z + w_z) dm (Eq. 10, last line) by Stokes (Eq. 11).  The
 * vertices (rotated frame) must be counter-clockwise.
 */
static double tri_visible_integral(const double v[3][2], double wx, double wz)
{
    double oa[3][2], ob[3][2];
    int alive[3], ca[3], cb[3];
    for (int k = 0; k < 3; ++k)
        alive[k] = clip_edge(v[k], v[(k + 1) % 3], wz, oa[k], ob[k], &ca[k], &cb[k]);
    double sum = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (!alive[k]) continue;
        sum += line_term(oa[k], ob[k], wx, wz);
        /* the next surviving edge in boundary order (possibly this one) */
        int nx = -1;
        for (int s = 1; s <= 3; ++s) {
            if (alive[(k + s) % 3]) { nx = (k + s) % 3; break; }
        }
        if (cb[k] || ca[nx]) sum += arc_term(ob[k], oa[nx]);
    }
    return sum;
}

/* Exported for the Stokes pin: one triangle, unrotated omega (unit, z > 0).
 * Returns the integral of max(m~ . w, 0) / m~_z over the normal triangle. */
double oracle_tri_integral(double n0x, double n0y, double n1x, double n1y,
                           double n2x, double n2y, double wx, double wy, double wz)
{
    double phi = atan2(wy, wx);
    double c = cos(phi), s = sin(phi);
    double wr = sqrt(wx * wx + wy * wy);
    double v[3][2] = {{c * n0x + s * n0y, -s * n0x + c * n0y},
                      {c * n1x + s * n1y, -s * n1x + c * n1y},
                      {c * n2x + s * n2y, -s * n2x + c * n2y}};
    double A2 = area2(v[0][0], v[0][1], v[1][0], v[1][1], v[2][0], v[2][1]);
    if (A2 < 0.0) {
        double t0 = v[1][0], t1 = v[1][1];
        v[1][0] = v[2][0]; v[1][1] = v[2][1];
        v[2][0] = t0; v[2][1] = t1;
    }
    return tri_visible_integral(v, wr, wz);
}

/*
 * P(w) for one footprint, Eq. 10: sum over triangles of
 * k_r(T) / (2 ||n(T)||) * integral over n+(T).  A triangle whose normal
 * triangle has |(n_b - n_a) x (n_c - n_a)| < 1e-12 has collapsed onto a
 * segment (or a point), where Eq. 10's ratio is 0/0; its contribution is
 * then the uv-space form of Eq. 13 over its uv triangle (see
 * collapsed_uv_form).
 */
/* max(m~ . w, 0) / m~_z */
static double visible_cos_ratio(double mx, double my, const double *w)
{
    double mz = sqrt(1.0 - mx * mx - my * my);
    double c = mx * w[0] + my * w[1] + mz * w[2];
    return (c > 0.0 ? c : 0.0) / mz;
}

/*
 * Eq. 13's uv-space integral over a uv triangle (area 1/2) whose normal
 * image is a segment: integral over T_uv of max(n~(u) . w, 0) / n~_z(u) du.
 * With P, Q the two farthest normal vertices and tau the position along
 * P -> Q, tau(u) is affine on the triangle, so a uniform point of the
 * triangle maps to the piecewise-linear (triangular) density on
 * [tau_1, tau_3] with its peak at tau_2 (the sorted vertex positions).  The
 * visible part of the segment is the interval Alg. 1 keeps; each linear
 * piece of the density is integrated over it by Gauss-Legendre (gl_x, gl_w
 * on [-1, 1], ngl points).
 */
static double collapsed_uv_form(const double *a, const double *b, const double *c, const double *w,
                                double c_phi, double s_phi, const double *gl_x, const double *gl_w, int ngl)
{
    const double *v[3] = {a, b, c};
    double best = -1.0;
    int ip = 0, iq = 1;
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j) {
            double dx = v[j][0] - v[i][0], dy = v[j][1] - v[i][1];
            double d2 = dx * dx + dy * dy;
            if (d2 > best) { best = d2; ip = i; iq = j; }
        }
    if (best == 0.0) return 0.5 * visible_cos_ratio(a[0], a[1], w);
    const double *P = v[ip], *Q = v[iq];
    double ex = Q[0] - P[0], ey = Q[1] - P[1];
    double tau[3];
    for (int i = 0; i < 3; ++i) tau[i] = ((v[i][0] - P[0]) * ex + (v[i][1] - P[1]) * ey) / best;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2 - i; ++j)
            if (tau[j] > tau[j + 1]) { double t = tau[j]; tau[j] = tau[j + 1]; tau[j + 1] = t; }
    /* visible interval of P -> Q from Alg. 1 in the rotated frame */
    double pr[2] = {c_phi * P[0] + s_phi * P[1], -s_phi * P[0] + c_phi * P[1]};
    double qr[2] = {c_phi * Q[0] + s_phi * Q[1], -s_phi * Q[0] + c_phi * Q[1]};
    double oa[2], ob[2];
    int ca, cb;
    if (!clip_edge(pr, qr, w[2], oa, ob, &ca, &cb)) return 0.0;
    double L2 = (qr[0] - pr[0]) * (qr[0] - pr[0]) + (qr[1] - pr[1]) * (qr[1] - pr[1]);
    double tlo = ((oa[0] - pr[0]) * (qr[0] - pr[0]) + (oa[1] - pr[1]) * (qr[1] - pr[1])) / L2;
    double thi = ((ob[0] - pr[0]) * (qr[0] - pr[0]) + (ob[1] - pr[1]) * (qr[1] - pr[1])) / L2;
    double span = tau[2] - tau[0];
    double sum = 0.0;
    for (int piece = 0; piece < 2; ++piece) {
        double t0 = tau[piece], t1 = tau[piece + 1];
        double lo = fmax(t0, tlo), hi = fmin(t1, thi);
        if (!(hi > lo) || t1 == t0) continue;
        for (int g = 0; g < ngl; ++g) {
            double t = 0.5 * (lo + hi) + 0.5 * (hi - lo) * gl_x[g];
            double dens = piece == 0 ? 2.0 * (t - t0) / (span * (t1 - t0)) : 2.0 * (t1 - t) / (span * (t1 - t0));
            sum += 0.5 * (hi - lo) * gl_w[g] * dens * visible_cos_ratio(P[0] + t * ex, P[1] + t * ey, w);
        }
    }
    return 0.5 * sum;
}

static double projarea_one(const double *st, int N, const double *qq, const double *w,
                           const double *gl_x, const double *gl_w, int ngl)
{
    double x = qq[0], y = qq[1], sxx = qq[2], sxy = qq[3], syy = qq[4];
    double det = sxx * syy - sxy * sxy;
    if (!(sxx > 0.0) || !(syy > 0.0) || !(det > 0.0)) return NAN;
    double ia = syy / det, ib = -sxy / det, ic = sxx / det;
    double norm = 1.0 / (2.0 * M_PI * sqrt(det));
    double wx = w[0], wy = w[1], wz = w[2];
    double phi = atan2(wy, wx);
    double c = cos(phi), s = sin(phi);
    double wr = sqrt(wx * wx + wy * wy);
    int i0, i1, j0, j1;
    quad_range(N, x, y, sxx, syy, &i0, &i1, &j0, &j1);
    double P = 0.0;
    for (int j = j0; j <= j1; ++j) {
        for (int i = i0; i <= i1; ++i) {
            double n[4][2];
            texel(st, N, i, j, n[0]);
            texel(st, N, i + 1, j, n[1]);
            texel(st, N, i, j + 1, n[2]);
            texel(st, N, i + 1, j + 1, n[3]);
            for (int tri = 0; tri < 2; ++tri) {
                static const int vid[2][3] = {{0, 1, 2}, {3, 2, 1}};
                /* uv centroid: (i + 1/3, j + 1/3) lower, (i + 2/3, j + 2/3) upper */
                double gx = i + (tri == 0 ? 1.0 / 3.0 : 2.0 / 3.0) - x;
                double gy = j + (tri == 0 ? 1.0 / 3.0 : 2.0 / 3.0) - y;
                double q = ia * gx * gx + 2.0 * ib * gx * gy + ic * gy * gy;
                if (q > ORACLE_QCUT) continue;
                double k = norm * exp(-0.5 * q);
                const double *a = n[vid[tri][0]], *b = n[vid[tri][1]], *cc = n[vid[tri][2]];
                double A2 = area2(a[0], a[1], b[0], b[1], cc[0], cc[1]);
                if (fabs(A2) < 1e-12) {
                    P += k * collapsed_uv_form(a, b, cc, w, c, s, gl_x, gl_w, ngl);
                    continue;
                }
                double v[3][2] = {{c * a[0] + s * a[1], -s * a[0] + c * a[1]},
                                  {c * b[0] + s * b[1], -s * b[0] + c * b[1]},
                                  {c * cc[0] + s * cc[1], -s * cc[0] + c * cc[1]}};
                if (A2 < 0.0) {
                    double t0 = v[1][0], t1 = v[1][1];
                    v[1][0] = v[2][0]; v[1][1] = v[2][1];
                    v[2][0] = t0; v[2][1] = t1;
                }
                P += k * tri_visible_integral(v, wr, wz) / fabs(A2);
            }
        }
    }
    return P;
}

void oracle_projarea(const double *st, int N, const double *q, const double *w,
                     int64_t k0, int64_t k1, double *P, const double *gl_x, const double *gl_w, int ngl)
{
    for (int64_t k = k0; k < k1; ++k) P[k] = projarea_one(st, N, q + 7 * k, w + 3 * k, gl_x, gl_w, ngl);
}
