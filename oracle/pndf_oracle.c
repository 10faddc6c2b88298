/*
 * FP64 CPU oracle for the position-normal-manifold P-NDF and the analytic
 * projected-area integral.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA path.  It is a plain,
 * slow, exhaustive evaluation: no hierarchy, no blocking, no reordering.
 * Every function is pinned by tests against closed forms, invariants, brute
 * force or quadrature (tests/test_oracle_*.py), and altered copies of it are
 * caught (tests/test_oracle_mutants.py): none is parity unpinned.
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

/*
 * Footprint kernels k_r(d), d = u - x, of Eq. 2 (the Gaussian of Sec. 5 and
 * the disk and box filters of the kernel ablation, which match a Gaussian's
 * (6 sigma)^2 footprint with a (3 sigma)^2 one), with S = [[sxx, sxy], [sxy,
 * syy]] and q = d^T S^-1 d:
 *   0 Gaussian: exp(-q/2) / (2 pi sqrt(det S)) where q <= 16, else 0;
 *   1 disk: 1 / (2.25 pi sqrt(det S)) where q <= 1.5^2, else 0;
 *   2 box: 1 / (9 sqrt(det S)) where |L^-1 d|_inf <= 1.5, S = L L^T (the
 *     Cholesky factor; for S = sigma^2 I the square of side 3 sigma).
 * Their supports' bounding-box half-widths (r_x, r_y): 4 (sqrt(sxx),
 * sqrt(syy)); 1.5 (sqrt(sxx), sqrt(syy)); 1.5 (l11, |l21| + l22).  All lie
 * inside the Gaussian's 4-sigma box.  A point within rounding of a disk or
 * box edge flags the query like a Gaussian cut tie.
 */
enum { OK_GAUSS = 0, OK_DISK = 1, OK_BOX = 2 };
#define ORACLE_SUPPORT_EPS 1e-5

static void kernel_halfwidths(int kernel, double sxx, double sxy, double syy, double *rx, double *ry)
{
    if (kernel == OK_GAUSS) {
        *rx = 4.0 * sqrt(sxx);
        *ry = 4.0 * sqrt(syy);
    } else if (kernel == OK_DISK) {
        *rx = 1.5 * sqrt(sxx);
        *ry = 1.5 * sqrt(syy);
    } else {
        double l11 = sqrt(sxx), l21 = sxy / l11, l22 = sqrt(syy - l21 * l21);
        *rx = 1.5 * l11;
        *ry = 1.5 * (fabs(l21) + l22);
    }
}

/* Disk or box weight at d (q = d^T S^-1 d given); 0 outside the support. */
static double flat_kernel(int kernel, double dx, double dy, double q, double sxx, double sxy, double syy,
                          double det, uint32_t *flags)
{
    if (kernel == OK_DISK) {
        if (fabs(q - 2.25) <= ORACLE_SUPPORT_EPS) *flags |= OF_NEAR_CUT;
        return q <= 2.25 ? 1.0 / (2.25 * M_PI * sqrt(det)) : 0.0;
    }
    double l11 = sqrt(sxx), l21 = sxy / l11, l22 = sqrt(syy - l21 * l21);
    double v1 = dx / l11, v2 = (dy - l21 * v1) / l22;
    double vm = fmax(fabs(v1), fabs(v2));
    if (fabs(vm - 1.5) <= ORACLE_SUPPORT_EPS) *flags |= OF_NEAR_CUT;
    return vm <= 1.5 ? 1.0 / (9.0 * sqrt(det)) : 0.0;
}

/*
 * Eq. 6 (Jacobian clamp): a fine triangle whose Jacobian |cross| is below eps
 * is replaced by an equilateral normal triangle of area eps / 2 (Jacobian
 * exactly eps), centred at the normal-space centroid of its three vertices,
 * with a fixed counter-clockwise orientation (vertex k at 90 + 120 k
 * degrees), its vertices taking the triangle's uv vertices in order.
 */
static void eqtri(const double *na, const double *nb, const double *nc, double eps, double E[3][2])
{
    double gx = (na[0] + nb[0] + nc[0]) / 3.0, gy = (na[1] + nb[1] + nc[1]) / 3.0;
    double side = sqrt(2.0 * eps / sqrt(3.0));  /* (sqrt(3) / 4) side^2 = eps / 2 */
    double rho = side / sqrt(3.0);              /* circumradius */
    for (int k = 0; k < 3; ++k) {
        double ang = M_PI / 2.0 + 2.0 * M_PI * k / 3.0;
        E[k][0] = gx + rho * cos(ang);
        E[k][1] = gy + rho * sin(ang);
    }
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
static void pndf_one(const double *st, int N, const double *qq, int kernel, double jac_eps,
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
                double E[3][2];
                if (jac_eps > 0.0 && fabs(A2) < jac_eps) {
                    /* Eq. 6: test the equilateral replacement (Jacobian eps) instead */
                    eqtri(na, nb, nc, jac_eps, E);
                    na = E[0]; nb = E[1]; nc = E[2];
                    A2 = area2(na[0], na[1], nb[0], nb[1], nc[0], nc[1]);
                }
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
                double J = fabs(A2);
                if (jac_eps > 0.0 && J < jac_eps) J = jac_eps;  /* the replacement's exact Jacobian */
                if (kernel != OK_GAUSS) {
                    double w = flat_kernel(kernel, dx, dy, q, sxx, sxy, syy, det, &flags);
                    if (w == 0.0) continue;
                    if (0.5 * J < ORACLE_TINY_AREA) flags |= OF_TINY;
                    D += w / J;
                    nh += 1;
                    hsum += fmix32((uint32_t)(2u * ((uint32_t)j * (uint32_t)(N - 1) + (uint32_t)i) + (uint32_t)tri));
                    continue;
                }
                if (fabs(q - ORACLE_QCUT) <= ORACLE_CUT_EPS) flags |= OF_NEAR_CUT;
                if (q > ORACLE_QCUT) continue;
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

/* Evaluate queries [k0, k1) with footprint kernel `kernel` (OK_*).  Safe to
 * call concurrently on disjoint ranges. */
void oracle_pndf(const double *st, int N, const double *q, int64_t k0, int64_t k1, int kernel, double jac_eps,
                 double *D, uint32_t *flags, int64_t *nhits, uint32_t *hsum)
{
    for (int64_t k = k0; k < k1; ++k)
        pndf_one(st, N, q + 7 * k, kernel, jac_eps, D + k, flags + k, nhits + k, hsum + k);
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

/*
 * App. B derives the clip ellipse (m_x / w_z)^2 + m_y^2 = 1 and the arc term
 * from w_x^2 + w_z^2 = 1 after the rotation, i.e. for a unit direction.  A
 * direction given in single precision is unit only to about 1e-8, and the
 * line terms (which use w as given) then disagree with the arc terms by that
 * relative amount, which is large against a triangle whose visible part is
 * small.  The direction is therefore taken as the unit vector w / |w|.
 */
static void unit_dir(const double *w_in, double w[3])
{
    double n = sqrt(w_in[0] * w_in[0] + w_in[1] * w_in[1] + w_in[2] * w_in[2]);
    w[0] = w_in[0] / n;
    w[1] = w_in[1] / n;
    w[2] = w_in[2] / n;
}

/* Exported for the Stokes pin: one triangle, unrotated omega (unit, z > 0).
 * Returns the integral of max(m~ . w, 0) / m~_z over the normal triangle. */
double oracle_tri_integral(double n0x, double n0y, double n1x, double n1y,
                           double n2x, double n2y, double wx_in, double wy_in, double wz_in)
{
    double w[3], w_in[3] = {wx_in, wy_in, wz_in};
    unit_dir(w_in, w);
    double wx = w[0], wy = w[1], wz = w[2];
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

static double projarea_one(const double *st, int N, const double *qq, const double *w_in,
                           const double *gl_x, const double *gl_w, int ngl)
{
    double w[3];
    unit_dir(w_in, w);
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

/* ------------------------------------------------------------------------- */
/* Cluster hierarchy and tau cut (Sec. 4.2 on mesh clustering, Eq. 7-8,     */
/* App. A).                                                                  */
/* ------------------------------------------------------------------------- */
/*
 * A node (l, I, J) covers the 2^l x 2^l quads [aI, aI + a) x [aJ, aJ + a),
 * a = 2^l, and uv square [aI, aI + a] x [aJ, aJ + a].  Its cluster is one
 * 1 x 1 grid of two triangles split like a quad (anti-diagonal), with corner
 * normals c00, c10, c01, c11 at uv (aI, aJ), (aI + a, aJ), (aI, aJ + a),
 * (aI + a, aJ + a): lower (c00, c10, c01), upper (c11, c01, c10).
 *
 * Eq. 7: the corner normals minimise
 *     F(c) = integral over the node of ||n^l(u) - n(u)||^2 / |det J(u)| du,
 * with n^l piecewise linear on the cluster triangles and n piecewise linear
 * on the fine triangles.  Every fine triangle lies inside one cluster
 * triangle, so the integrand is a quadratic on each fine triangle and the
 * three-point edge-midpoint rule integrates it exactly.  |det J| on a fine
 * triangle is its |cross|; Eq. 6 clamps the Jacobian at 1e-6, and the weight
 * 1 / max(|cross|, 1e-6) uses the same clamp so that flat triangles stay
 * finite.  The residual e^l of Eq. 8 is read as the 2-norm of the weighted
 * approximation error at the optimum, sqrt(F(c*)) (the printed norm of the
 * normal-equation residual is zero at the optimum); sqrt(F) has units of
 * texel^2, like r_x r_y, so tau is dimensionless.
 *
 * Readings: clusters exist at levels >= 2 (the 4 x 4-quad block and above)
 * and only for nodes whose quads all lie inside the map; the cut is taken top
 * down from the query's entry nodes (the level-l nodes meeting the 4-sigma
 * box, l = the smallest level >= 2 with 2^l >= max(r_x, r_y), at most the top
 * level), and a node is a cluster when e^l <= r_x r_y tau with r_x = 4
 * sqrt(Sigma_xx), r_y = 4 sqrt(Sigma_yy).  The cut depends on the footprint
 * only, not on m, so D with clusters is the P-NDF of a piecewise-linear
 * surrogate map; a node that is not cut is replaced by its children, and a
 * level-2 node that is not cut by its exact triangles (Eq. 5).
 */
#define ORACLE_JAC_EPS 1e-6
#define ORACLE_TAU_EPS 1e-5     /* residual vs r_x r_y tau (FP32 storage and FP32 threshold) */
#define ORACLE_RADIUS_EPS 3e-5  /* entry radius vs 2^l (FP32 square root, inflated box) */

enum { OF_NEAR_TAU = 32u };  /* a cut decision within rounding of its threshold */

static int top_level_of(int N)
{
    int L = 0;
    while ((1 << L) < N - 1) ++L;
    return L < 2 ? 2 : L;
}

/* Hat functions of the cluster at normalised local coordinates (s, t). */
static void cluster_basis(double s, double t, int upper, double phi[4])
{
    if (!upper) {
        phi[0] = 1.0 - s - t; phi[1] = s; phi[2] = t; phi[3] = 0.0;
    } else {
        phi[0] = 0.0; phi[1] = 1.0 - t; phi[2] = 1.0 - s; phi[3] = s + t - 1.0;
    }
}

/* Solve G x = R (4 x 4, two right-hand sides) by Gaussian elimination with
 * partial pivoting.  Returns 0 if G is singular. */
static int solve4(double G[4][4], double R[4][2], double x[4][2])
{
    for (int k = 0; k < 4; ++k) {
        int p = k;
        for (int r = k + 1; r < 4; ++r)
            if (fabs(G[r][k]) > fabs(G[p][k])) p = r;
        if (G[p][k] == 0.0) return 0;
        if (p != k) {
            for (int c = 0; c < 4; ++c) { double tmp = G[k][c]; G[k][c] = G[p][c]; G[p][c] = tmp; }
            for (int c = 0; c < 2; ++c) { double tmp = R[k][c]; R[k][c] = R[p][c]; R[p][c] = tmp; }
        }
        for (int r = k + 1; r < 4; ++r) {
            double f = G[r][k] / G[k][k];
            for (int c = k; c < 4; ++c) G[r][c] -= f * G[k][c];
            for (int c = 0; c < 2; ++c) R[r][c] -= f * R[k][c];
        }
    }
    for (int k = 3; k >= 0; --k)
        for (int c = 0; c < 2; ++c) {
            double v = R[k][c];
            for (int j = k + 1; j < 4; ++j) v -= G[k][j] * x[j][c];
            x[k][c] = v / G[k][k];
        }
    return 1;
}

/* The fine triangles of quad (i, j): uv vertices and normals, Tab. 1 order. */
static void quad_tri(const double *st, int N, int i, int j, int tri, double uv[3][2], double nv[3][2])
{
    static const int lower[3][2] = {{0, 0}, {1, 0}, {0, 1}};
    static const int upper[3][2] = {{1, 1}, {0, 1}, {1, 0}};
    const int (*v)[2] = tri ? upper : lower;
    for (int k = 0; k < 3; ++k) {
        uv[k][0] = i + v[k][0];
        uv[k][1] = j + v[k][1];
        texel(st, N, i + v[k][0], j + v[k][1], nv[k]);
    }
}

/* Weighted quadrature points of the fine triangles of node (l, I, J): calls
 * fn(ctx, s, t, upper, n, weight) for each edge midpoint, with weight =
 * (area / 3) / max(|cross|, eps). */
typedef void (*midpoint_fn)(void *ctx, double s, double t, int upper, const double n[2], double w);

static void node_midpoints(const double *st, int N, int l, int I, int J, midpoint_fn fn, void *ctx)
{
    int a = 1 << l;
    for (int j = a * J; j < a * J + a; ++j)
        for (int i = a * I; i < a * I + a; ++i)
            for (int tri = 0; tri < 2; ++tri) {
                double uv[3][2], nv[3][2];
                quad_tri(st, N, i, j, tri, uv, nv);
                double cr = fabs(area2(nv[0][0], nv[0][1], nv[1][0], nv[1][1], nv[2][0], nv[2][1]));
                double w = (0.5 / 3.0) / fmax(cr, ORACLE_JAC_EPS);
                /* which cluster triangle holds this fine triangle: its centroid */
                double cs = ((uv[0][0] + uv[1][0] + uv[2][0]) / 3.0 - a * I) / a;
                double ct = ((uv[0][1] + uv[1][1] + uv[2][1]) / 3.0 - a * J) / a;
                int upper = cs + ct > 1.0;
                for (int k = 0; k < 3; ++k) {
                    int k2 = (k + 1) % 3;
                    double s = (0.5 * (uv[k][0] + uv[k2][0]) - a * I) / a;
                    double t = (0.5 * (uv[k][1] + uv[k2][1]) - a * J) / a;
                    double n[2] = {0.5 * (nv[k][0] + nv[k2][0]), 0.5 * (nv[k][1] + nv[k2][1])};
                    fn(ctx, s, t, upper, n, w);
                }
            }
}

struct normal_eq { double G[4][4], R[4][2]; };

static void add_normal_eq(void *ctx, double s, double t, int upper, const double n[2], double w)
{
    struct normal_eq *ne = (struct normal_eq *)ctx;
    double phi[4];
    cluster_basis(s, t, upper, phi);
    for (int r = 0; r < 4; ++r) {
        for (int c = 0; c < 4; ++c) ne->G[r][c] += w * phi[r] * phi[c];
        ne->R[r][0] += w * phi[r] * n[0];
        ne->R[r][1] += w * phi[r] * n[1];
    }
}

struct misfit { const double *c; double F; };

static void add_misfit(void *ctx, double s, double t, int upper, const double n[2], double w)
{
    struct misfit *mf = (struct misfit *)ctx;
    double phi[4];
    cluster_basis(s, t, upper, phi);
    double dx = -n[0], dy = -n[1];
    for (int a = 0; a < 4; ++a) {
        dx += phi[a] * mf->c[2 * a];
        dy += phi[a] * mf->c[2 * a + 1];
    }
    mf->F += w * (dx * dx + dy * dy);
}

/*
 * Eq. 7-8 for node (l, I, J): corner normals c = (c00, c10, c01, c11) as
 * (s, t) pairs and e = sqrt(F(c)).  Returns 0 (c and e untouched) when the node is
 * not entirely inside the map or the normal equations are singular.
 */
int oracle_cluster_fit(const double *st, int N, int l, int I, int J, double *c, double *e)
{
    int a = 1 << l;
    if (a * (I + 1) > N - 1 || a * (J + 1) > N - 1) return 0;
    struct normal_eq ne;
    memset(&ne, 0, sizeof ne);
    node_midpoints(st, N, l, I, J, add_normal_eq, &ne);
    double x[4][2];
    if (!solve4(ne.G, ne.R, x)) return 0;
    for (int k = 0; k < 4; ++k) { c[2 * k] = x[k][0]; c[2 * k + 1] = x[k][1]; }
    struct misfit mf = {c, 0.0};
    node_midpoints(st, N, l, I, J, add_misfit, &mf);
    *e = sqrt(mf.F);
    return 1;
}

/* Pyramid layout of the precomputed fits: levels 2..L, level l holds
 * S_l x S_l nodes (S_l = 2^(L - l)) row-major by (J, I). */
static size_t cluster_offset(int L, int l)
{
    size_t off = 0;
    for (int k = 2; k < l; ++k) off += ((size_t)1 << (L - k)) * ((size_t)1 << (L - k));
    return off;
}

/* Fits of level-l nodes in rows [J0, J1): c (8 per node) and e (1 per node,
 * +inf where no cluster exists).  Safe on disjoint row ranges. */
void oracle_cluster_build(const double *st, int N, int l, int J0, int J1, double *c_all, double *e_all)
{
    int L = top_level_of(N);
    size_t S = (size_t)1 << (L - l), off = cluster_offset(L, l);
    for (int J = J0; J < J1; ++J)
        for (size_t I = 0; I < S; ++I) {
            size_t k = off + (size_t)J * S + I;
            if (!oracle_cluster_fit(st, N, l, (int)I, J, c_all + 8 * k, e_all + k)) {
                for (int t = 0; t < 8; ++t) c_all[8 * k + t] = 0.0;
                e_all[k] = INFINITY;
            }
        }
}

/*
 * Normal hull of every node at levels 2..L (smin, tmin, smax, tmax; 4 per
 * node, same layout as the fits): the box of the normals of all texels its
 * quads touch, of its own cluster corners and of its children's hulls.  Any
 * piece of any cut below a node (exact triangle or cluster triangle) lies in
 * its hull, so where m is outside it the node's cut decision cannot change D.
 * Sequential (one call for the whole pyramid).
 */
void oracle_cluster_hulls(const double *st, int N, const double *c_all, const double *e_all, double *hull)
{
    int L = top_level_of(N);
    for (int l = 2; l <= L; ++l) {
        size_t S = (size_t)1 << (L - l), off = cluster_offset(L, l);
        int a = 1 << l;
        for (size_t J = 0; J < S; ++J)
            for (size_t I = 0; I < S; ++I) {
                size_t k = off + J * S + I;
                double *h = hull + 4 * k;
                h[0] = h[1] = INFINITY;
                h[2] = h[3] = -INFINITY;
                if (l == 2) {
                    for (int j = (int)(a * J); j <= (int)(a * J) + a && j <= N - 1; ++j)
                        for (int i = (int)(a * I); i <= (int)(a * I) + a && i <= N - 1; ++i) {
                            if (i > N - 1 || j > N - 1) continue;
                            if ((int)(a * I) > N - 2 || (int)(a * J) > N - 2) continue;  /* node has no quad */
                            double n[2];
                            texel(st, N, i, j, n);
                            h[0] = fmin(h[0], n[0]); h[1] = fmin(h[1], n[1]);
                            h[2] = fmax(h[2], n[0]); h[3] = fmax(h[3], n[1]);
                        }
                } else {
                    size_t Sc = S * 2, offc = cluster_offset(L, l - 1);
                    for (int dj = 0; dj < 2; ++dj)
                        for (int di = 0; di < 2; ++di) {
                            const double *g = hull + 4 * (offc + (2 * J + dj) * Sc + 2 * I + di);
                            h[0] = fmin(h[0], g[0]); h[1] = fmin(h[1], g[1]);
                            h[2] = fmax(h[2], g[2]); h[3] = fmax(h[3], g[3]);
                        }
                }
                if (isfinite(e_all[k]))
                    for (int t = 0; t < 4; ++t) {
                        const double *c = c_all + 8 * k + 2 * t;
                        h[0] = fmin(h[0], c[0]); h[1] = fmin(h[1], c[1]);
                        h[2] = fmax(h[2], c[0]); h[3] = fmax(h[3], c[1]);
                    }
            }
    }
}

struct cl_query {
    const double *st, *c_all, *e_all, *hull;
    int N, L, kernel;
    double x, y, ia, ib, ic, norm, mx, my, rx, ry, theta, sxx, sxy, syy, det;
    double D;
    uint32_t flags, hsum;
    int64_t nh;
};

/* Test m against one triangle (uv a, b, c; normals na, nb, nc) whose map
 * u -> n has Jacobian |cross| / scale^2 (Eq. 4), accumulating Eq. 5. */
static void cl_triangle(struct cl_query *Q, const double uv[3][2], const double nv[3][2], double scale, uint32_t id)
{
    double mx = Q->mx, my = Q->my;
    double A2 = area2(nv[0][0], nv[0][1], nv[1][0], nv[1][1], nv[2][0], nv[2][1]);
    double lox = fmin(nv[0][0], fmin(nv[1][0], nv[2][0])) - ORACLE_EDGE_EPS;
    double hix = fmax(nv[0][0], fmax(nv[1][0], nv[2][0])) + ORACLE_EDGE_EPS;
    double loy = fmin(nv[0][1], fmin(nv[1][1], nv[2][1])) - ORACLE_EDGE_EPS;
    double hiy = fmax(nv[0][1], fmax(nv[1][1], nv[2][1])) + ORACLE_EDGE_EPS;
    if (mx >= lox && mx <= hix && my >= loy && my <= hiy) {
        double dmin = seg_dist(mx, my, nv[0][0], nv[0][1], nv[1][0], nv[1][1]);
        dmin = fmin(dmin, seg_dist(mx, my, nv[1][0], nv[1][1], nv[2][0], nv[2][1]));
        dmin = fmin(dmin, seg_dist(mx, my, nv[2][0], nv[2][1], nv[0][0], nv[0][1]));
        if (dmin <= ORACLE_EDGE_EPS) Q->flags |= (A2 == 0.0) ? (OF_NEAR_EDGE | OF_DEGENERATE) : OF_NEAR_EDGE;
    }
    if (A2 == 0.0) return;
    double l0 = area2(mx, my, nv[1][0], nv[1][1], nv[2][0], nv[2][1]) / A2;
    double l1 = area2(nv[0][0], nv[0][1], mx, my, nv[2][0], nv[2][1]) / A2;
    double l2 = area2(nv[0][0], nv[0][1], nv[1][0], nv[1][1], mx, my) / A2;
    if (!(l0 >= 0.0 && l1 >= 0.0 && l2 >= 0.0)) return;
    double ux = uv[0][0] * l0 + uv[1][0] * l1 + uv[2][0] * l2;
    double uy = uv[0][1] * l0 + uv[1][1] * l1 + uv[2][1] * l2;
    double dx = ux - Q->x, dy = uy - Q->y;
    double q = Q->ia * dx * dx + 2.0 * Q->ib * dx * dy + Q->ic * dy * dy;
    double J = fabs(A2) / (scale * scale);
    double w;
    if (Q->kernel != OK_GAUSS) {
        w = flat_kernel(Q->kernel, dx, dy, q, Q->sxx, Q->sxy, Q->syy, Q->det, &Q->flags);
        if (w == 0.0) return;
    } else {
        if (fabs(q - ORACLE_QCUT) <= ORACLE_CUT_EPS) Q->flags |= OF_NEAR_CUT;
        if (q > ORACLE_QCUT) return;
        w = Q->norm * exp(-0.5 * q);
    }
    if (0.5 * fabs(A2) < ORACLE_TINY_AREA) Q->flags |= OF_TINY;
    Q->D += w / J;
    Q->nh += 1;
    Q->hsum += fmix32(id);
}

static int near_threshold(double v, double thr, double eps)
{
    return fabs(v - thr) <= eps * fmax(fabs(thr), 1e-300);
}

static void cl_visit(struct cl_query *Q, int l, int I, int J)
{
    int a = 1 << l, N = Q->N;
    if (a * I > N - 2 || a * J > N - 2) return;  /* no quad of this node exists */
    /* no content within the 4-sigma box: contributes k_r = 0 (Eq. 5) */
    if (a * I > Q->x + Q->rx || a * (I + 1) < Q->x - Q->rx || a * J > Q->y + Q->ry || a * (J + 1) < Q->y - Q->ry)
        return;
    size_t S = (size_t)1 << (Q->L - l);
    size_t k = cluster_offset(Q->L, l) + (size_t)J * S + (size_t)I;
    double e = Q->e_all[k];
    if (Q->theta > 0.0 && isfinite(e)) {
        /* a close call matters only where m can meet the node's pieces */
        const double *h = Q->hull + 4 * k;
        if (near_threshold(e, Q->theta, ORACLE_TAU_EPS) && Q->mx >= h[0] - ORACLE_EDGE_EPS && Q->mx <= h[2] + ORACLE_EDGE_EPS &&
            Q->my >= h[1] - ORACLE_EDGE_EPS && Q->my <= h[3] + ORACLE_EDGE_EPS)
            Q->flags |= OF_NEAR_TAU;
        if (e <= Q->theta) {
            const double *c = Q->c_all + 8 * k;
            double ox = a * I, oy = a * J;
            double uv0[3][2] = {{ox, oy}, {ox + a, oy}, {ox, oy + a}};
            double nv0[3][2] = {{c[0], c[1]}, {c[2], c[3]}, {c[4], c[5]}};
            double uv1[3][2] = {{ox + a, oy + a}, {ox, oy + a}, {ox + a, oy}};
            double nv1[3][2] = {{c[6], c[7]}, {c[4], c[5]}, {c[2], c[3]}};
            uint32_t id = 0x80000000u | ((uint32_t)l << 27) | ((uint32_t)((size_t)J * S + (size_t)I) << 1);
            cl_triangle(Q, uv0, nv0, (double)a, id);
            cl_triangle(Q, uv1, nv1, (double)a, id | 1u);
            return;
        }
    }
    if (l == 2) {
        for (int j = a * J; j < a * J + a && j <= N - 2; ++j)
            for (int i = a * I; i < a * I + a && i <= N - 2; ++i)
                for (int tri = 0; tri < 2; ++tri) {
                    double uv[3][2], nv[3][2];
                    quad_tri(Q->st, N, i, j, tri, uv, nv);
                    cl_triangle(Q, uv, nv, 1.0, (uint32_t)(2u * ((uint32_t)j * (uint32_t)(N - 1) + (uint32_t)i) + (uint32_t)tri));
                }
        return;
    }
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) cl_visit(Q, l - 1, 2 * I + di, 2 * J + dj);
}

static void pndf_cluster_one(const double *st, int N, const double *qq, int kernel, double tau,
                             const double *c_all, const double *e_all, const double *hull, double *D_out,
                             uint32_t *flags_out, int64_t *nhits_out, uint32_t *hash_out)
{
    double sxx = qq[2], sxy = qq[3], syy = qq[4];
    double det = sxx * syy - sxy * sxy;
    if (!(sxx > 0.0) || !(syy > 0.0) || !(det > 0.0)) {
        *D_out = NAN;
        *flags_out = OF_INVALID;
        *nhits_out = 0;
        *hash_out = 0;
        return;
    }
    struct cl_query Q;
    memset(&Q, 0, sizeof Q);
    Q.st = st; Q.c_all = c_all; Q.e_all = e_all; Q.hull = hull; Q.N = N; Q.L = top_level_of(N);
    Q.x = qq[0]; Q.y = qq[1]; Q.mx = qq[5]; Q.my = qq[6];
    Q.ia = syy / det; Q.ib = -sxy / det; Q.ic = sxx / det;
    Q.norm = 1.0 / (2.0 * M_PI * sqrt(det));
    Q.kernel = kernel;
    Q.sxx = sxx; Q.sxy = sxy; Q.syy = syy; Q.det = det;
    kernel_halfwidths(kernel, sxx, sxy, syy, &Q.rx, &Q.ry);
    Q.theta = Q.rx * Q.ry * tau;
    /* entry level: smallest l >= 2 with 2^l >= max(r_x, r_y), at most L */
    double r = fmax(Q.rx, Q.ry);
    int le = 2;
    while (le < Q.L && (double)(1 << le) < r) ++le;
    for (int k = 2; k <= Q.L && tau > 0.0; ++k)
        if (near_threshold(r, (double)(1 << k), ORACLE_RADIUS_EPS)) Q.flags |= OF_NEAR_TAU;
    int a = 1 << le;
    int I0 = (int)fmax(ceil((Q.x - Q.rx) / a) - 1.0, 0.0), I1 = (int)fmin(floor((Q.x + Q.rx) / a), (double)((1 << (Q.L - le)) - 1));
    int J0 = (int)fmax(ceil((Q.y - Q.ry) / a) - 1.0, 0.0), J1 = (int)fmin(floor((Q.y + Q.ry) / a), (double)((1 << (Q.L - le)) - 1));
    for (int J = J0; J <= J1; ++J)
        for (int I = I0; I <= I1; ++I) cl_visit(&Q, le, I, J);
    *D_out = Q.D;
    *flags_out = Q.flags;
    *nhits_out = Q.nh;
    *hash_out = Q.hsum;
}

/* P-NDF with the cluster cut for queries [k0, k1) (footprint kernel as in
 * oracle_pndf; r_x, r_y of the cut are its support half-widths); tau <= 0 cuts nothing
 * (exact D, summed in traversal order).  c_all / e_all come from
 * oracle_cluster_build for every level 2..L, hull from oracle_cluster_hulls. */
void oracle_pndf_cluster(const double *st, int N, const double *q, int64_t k0, int64_t k1, int kernel, double tau,
                         const double *c_all, const double *e_all, const double *hull, double *D, uint32_t *flags,
                         int64_t *nhits, uint32_t *hsum)
{
    for (int64_t k = k0; k < k1; ++k)
        pndf_cluster_one(st, N, q + 7 * k, kernel, tau, c_all, e_all, hull, D + k, flags + k, nhits + k, hsum + k);
}

/*
 * P-NDF sampling (Sec. 3, Eq. 6): u ~ k_r(u - x) by the inverse CDF of the
 * caller's uniforms (U1, U2) in the whitened frame v, u = x + L v (S = L L^T):
 *   Gaussian cut at q = 16: |v|^2 = -2 ln(1 - U1 (1 - e^-8)), angle 2 pi U2;
 *   disk: |v| = 1.5 sqrt(U1), angle 2 pi U2;   box: v = 1.5 (2 U1 - 1, 2 U2 - 1);
 * then m = n(u) by Eq. 3 (the fine triangle holding u, barycentric), or the
 * same barycentric point of the Eq. 6 replacement when jac_eps > 0 and the
 * triangle's Jacobian is below it.  Flags per sample: 16 invalid S, 64 u
 * outside the map (m = 0), 1 u within 1e-9 texel of a quad or diagonal edge
 * (the triangle choice is a tie).  tri receives the triangle id (or -1).
 */
enum { OF_OUTSIDE = 64u };

void oracle_sample(const double *st, int N, const double *q, const double *U, int64_t k0, int64_t k1, int kernel,
                   double jac_eps, double *m_out, int64_t *tri_out, uint32_t *flags_out)
{
    for (int64_t k = k0; k < k1; ++k) {
        const double *qq = q + 7 * k;
        double x = qq[0], y = qq[1], sxx = qq[2], sxy = qq[3], syy = qq[4];
        double det = sxx * syy - sxy * sxy;
        double *m = m_out + 2 * k;
        m[0] = m[1] = 0.0;
        tri_out[k] = -1;
        flags_out[k] = 0;
        if (!(sxx > 0.0) || !(syy > 0.0) || !(det > 0.0)) {
            flags_out[k] = OF_INVALID;
            continue;
        }
        double u1 = U[2 * k], u2 = U[2 * k + 1], v1, v2;
        if (kernel == OK_BOX) {
            v1 = 1.5 * (2.0 * u1 - 1.0);
            v2 = 1.5 * (2.0 * u2 - 1.0);
        } else {
            double r = kernel == OK_DISK ? 1.5 * sqrt(u1) : sqrt(-2.0 * log(1.0 - u1 * (1.0 - exp(-8.0))));
            v1 = r * cos(2.0 * M_PI * u2);
            v2 = r * sin(2.0 * M_PI * u2);
        }
        double l11 = sqrt(sxx), l21 = sxy / l11, l22 = sqrt(syy - l21 * l21);
        double ux = x + l11 * v1, uy = y + l21 * v1 + l22 * v2;
        double fi = floor(ux), fj = floor(uy);
        if (!(fi >= 0.0 && fj >= 0.0 && fi <= N - 2 && fj <= N - 2)) {
            flags_out[k] = OF_OUTSIDE;
            continue;
        }
        int i = (int)fi, j = (int)fj;
        double fu = ux - fi, fv = uy - fj;
        const double tie = 1e-9;
        if (fu < tie || fu > 1.0 - tie || fv < tie || fv > 1.0 - tie || fabs(fu + fv - 1.0) < tie)
            flags_out[k] |= OF_NEAR_EDGE;
        int tri = fu + fv < 1.0 ? 0 : 1;
        double uv[3][2], nv[3][2], lam[3];
        quad_tri(st, N, i, j, tri, uv, nv);
        if (tri == 0) {
            lam[0] = 1.0 - fu - fv; lam[1] = fu; lam[2] = fv;
        } else {
            lam[0] = fu + fv - 1.0; lam[1] = 1.0 - fu; lam[2] = 1.0 - fv;
        }
        double A2 = area2(nv[0][0], nv[0][1], nv[1][0], nv[1][1], nv[2][0], nv[2][1]);
        if (jac_eps > 0.0 && fabs(A2) < jac_eps) {
            double E[3][2];
            eqtri(nv[0], nv[1], nv[2], jac_eps, E);
            for (int c = 0; c < 2; ++c) m[c] = lam[0] * E[0][c] + lam[1] * E[1][c] + lam[2] * E[2][c];
        } else {
            for (int c = 0; c < 2; ++c) m[c] = lam[0] * nv[0][c] + lam[1] * nv[1][c] + lam[2] * nv[2][c];
        }
        tri_out[k] = 2 * ((int64_t)j * (N - 1) + i) + tri;
    }
}

/* ------------------------------------------------------------------------- */
/* GGX projected-area fit per mip node (Eq. 12) and shadow-masking (Sec. 4.3) */
/* ------------------------------------------------------------------------- */
/*
 * Readings.  Eq. 12 with its parentheses restored (the printed form drops
 * them): P'(w) = (w_z + sqrt(w_z^2 + w_xy^T Omega w_xy)) / 2, the GGX
 * projected area (Lambda' = P'/w_z - 1 is the GGX Smith Lambda).  A mip node
 * (level l, 2^l x 2^l quads) is filtered by the box over its own quads (k =
 * 4^-l per unit uv area), for which Eq. 9-11 are exact.  Its P is taken at K
 * given unit directions; each gives a_k = (2 P_k - w_z)^2 - w_z^2 =
 * w_xy^T Omega w_xy, linear in (O_xx, O_xy, O_yy), solved by least squares
 * (the normal equations).  Only nodes whose quads all lie in the map are
 * fitted.  Inference blends the fits of the two mip levels around
 * lambda = log2(sqrt(12) max(sqrt(S_xx), sqrt(S_yy))) (a box of width b has
 * the variance b^2 / 12), each bilinear between node centres (nodes without a
 * fit drop out and the weights renormalise), lambda clamped to [2, L].
 * Shadow-masking, height-correlated form: G = H(m~.wi) H(m~.wo) /
 * (1 + Lambda(wi) + Lambda(wo)).
 */

/* One triangle's V_T / |cross| (Eq. 10-11, Alg. 1; uv form when collapsed). */
static double tri_ratio(const double *a, const double *b, const double *cc, const double *w_in,
                        const double *gl_x, const double *gl_w, int ngl)
{
    double w[3];
    unit_dir(w_in, w);
    double wx = w[0], wy = w[1], wz = w[2];
    double phi = atan2(wy, wx), c = cos(phi), s = sin(phi), wr = sqrt(wx * wx + wy * wy);
    double A2 = area2(a[0], a[1], b[0], b[1], cc[0], cc[1]);
    if (fabs(A2) < 1e-12) return collapsed_uv_form(a, b, cc, w, c, s, gl_x, gl_w, ngl);
    double v[3][2] = {{c * a[0] + s * a[1], -s * a[0] + c * a[1]},
                      {c * b[0] + s * b[1], -s * b[0] + c * b[1]},
                      {c * cc[0] + s * cc[1], -s * cc[0] + c * cc[1]}};
    if (A2 < 0.0) {
        double t0 = v[1][0], t1 = v[1][1];
        v[1][0] = v[2][0]; v[1][1] = v[2][1];
        v[2][0] = t0; v[2][1] = t1;
    }
    return tri_visible_integral(v, wr, wz) / fabs(A2);
}

/* Box-filtered projected area of node (l, I, J) at K directions (3 per):
 * P[k] = 4^-l sum over its triangles of V_T / |cross|.  0 if the node has a
 * quad outside the map. */
int oracle_ggx_node_P(const double *st, int N, int l, int I, int J, const double *dirs, int K,
                      const double *gl_x, const double *gl_w, int ngl, double *P)
{
    int a = 1 << l;
    if (a * (I + 1) > N - 1 || a * (J + 1) > N - 1) return 0;
    for (int k = 0; k < K; ++k) P[k] = 0.0;
    for (int j = a * J; j < a * J + a; ++j)
        for (int i = a * I; i < a * I + a; ++i)
            for (int tri = 0; tri < 2; ++tri) {
                double uv[3][2], nv[3][2];
                quad_tri(st, N, i, j, tri, uv, nv);
                for (int k = 0; k < K; ++k) P[k] += tri_ratio(nv[0], nv[1], nv[2], dirs + 3 * k, gl_x, gl_w, ngl);
            }
    for (int k = 0; k < K; ++k) P[k] /= (double)a * (double)a;
    return 1;
}

/* Least-squares Omega (O_xx, O_xy, O_yy) from P at K directions.  0 if the
 * normal equations are singular. */
int oracle_ggx_fit(const double *P, const double *dirs, int K, double *Omega)
{
    double A[3][3] = {{0}}, r[3] = {0};
    for (int k = 0; k < K; ++k) {
        double wx = dirs[3 * k], wy = dirs[3 * k + 1], wz = dirs[3 * k + 2];
        double t = 2.0 * P[k] - wz;
        double ak = t * t - wz * wz;
        double row[3] = {wx * wx, 2.0 * wx * wy, wy * wy};
        for (int p = 0; p < 3; ++p) {
            r[p] += row[p] * ak;
            for (int q = 0; q < 3; ++q) A[p][q] += row[p] * row[q];
        }
    }
    /* Gaussian elimination with partial pivoting */
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int p = c + 1; p < 3; ++p)
            if (fabs(A[p][c]) > fabs(A[piv][c])) piv = p;
        if (A[piv][c] == 0.0) return 0;
        if (piv != c) {
            for (int q = 0; q < 3; ++q) { double t = A[c][q]; A[c][q] = A[piv][q]; A[piv][q] = t; }
            double t = r[c]; r[c] = r[piv]; r[piv] = t;
        }
        for (int p = c + 1; p < 3; ++p) {
            double f = A[p][c] / A[c][c];
            for (int q = c; q < 3; ++q) A[p][q] -= f * A[c][q];
            r[p] -= f * r[c];
        }
    }
    for (int c = 2; c >= 0; --c) {
        double v = r[c];
        for (int q = c + 1; q < 3; ++q) v -= A[c][q] * Omega[q];
        Omega[c] = v / A[c][c];
    }
    return 1;
}

/* Fits of level-l nodes in rows [J0, J1) into Omega_all (3 per node, the
 * cluster layout of levels 2..L; NaN where the node has no fit). */
void oracle_ggx_build(const double *st, int N, int l, int J0, int J1, const double *dirs, int K,
                      const double *gl_x, const double *gl_w, int ngl, double *Omega_all)
{
    int L = top_level_of(N);
    size_t S = (size_t)1 << (L - l), off = cluster_offset(L, l);
    double P[64];
    for (int J = J0; J < J1; ++J)
        for (size_t I = 0; I < S; ++I) {
            double *O = Omega_all + 3 * (off + (size_t)J * S + I);
            if (K > 64 || !oracle_ggx_node_P(st, N, l, (int)I, J, dirs, K, gl_x, gl_w, ngl, P) ||
                !oracle_ggx_fit(P, dirs, K, O))
                O[0] = O[1] = O[2] = NAN;
        }
}

/* Omega at a footprint (x, y, S) by the blend described above; 0 if no node
 * contributes. */
static int ggx_omega_at(const double *Omega_all, int N, double x, double y, double sxx, double syy, double O[3])
{
    int L = top_level_of(N);
    double lam = log2(sqrt(12.0) * fmax(sqrt(sxx), sqrt(syy)));
    if (lam < 2.0) lam = 2.0;
    if (lam > L) lam = L;
    int l0 = (int)floor(lam), l1 = l0 < L ? l0 + 1 : l0;
    double tl = lam - l0;
    double acc[3] = {0, 0, 0}, wsum = 0.0;
    for (int side = 0; side < 2; ++side) {
        int l = side ? l1 : l0;
        double wl = side ? tl : 1.0 - tl;
        if (wl == 0.0) continue;
        double a = (double)(1 << l);
        int S = 1 << (L - l);
        double fx = x / a - 0.5, fy = y / a - 0.5;
        int i0 = (int)floor(fx), j0 = (int)floor(fy);
        double tx = fx - i0, ty = fy - j0;
        double lacc[3] = {0, 0, 0}, lw = 0.0;
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                int I = i0 + di, Jn = j0 + dj;
                if (I < 0) I = 0;
                if (I > S - 1) I = S - 1;
                if (Jn < 0) Jn = 0;
                if (Jn > S - 1) Jn = S - 1;
                const double *Ok = Omega_all + 3 * (cluster_offset(L, l) + (size_t)Jn * S + I);
                if (!isfinite(Ok[0])) continue;
                double w = (di ? tx : 1.0 - tx) * (dj ? ty : 1.0 - ty);
                for (int c = 0; c < 3; ++c) lacc[c] += w * Ok[c];
                lw += w;
            }
        if (lw > 0.0) {
            for (int c = 0; c < 3; ++c) acc[c] += wl * lacc[c] / lw;
            wsum += wl;
        }
    }
    if (!(wsum > 0.0)) return 0;
    for (int c = 0; c < 3; ++c) O[c] = acc[c] / wsum;
    return 1;
}

static double ggx_P(const double O[3], const double *w)
{
    double q = O[0] * w[0] * w[0] + 2.0 * O[1] * w[0] * w[1] + O[2] * w[1] * w[1];
    return 0.5 * (w[2] + sqrt(fmax(w[2] * w[2] + q, 0.0)));
}

/* Lambda'(w) = P'(w) / w_z - 1 per query (7 doubles) and direction (3);
 * NaN where no fit covers the footprint. */
void oracle_ggx_lambda(const double *Omega_all, int N, const double *q, const double *w, int64_t k0, int64_t k1,
                       double *lam)
{
    for (int64_t k = k0; k < k1; ++k) {
        double O[3];
        const double *qq = q + 7 * k;
        if (!ggx_omega_at(Omega_all, N, qq[0], qq[1], qq[2], qq[4], O)) {
            lam[k] = NAN;
            continue;
        }
        lam[k] = ggx_P(O, w + 3 * k) / w[3 * k + 2] - 1.0;
    }
}

/* Height-correlated shadow-masking G(wi, wo, m) with the GGX Lambda', m =
 * the query normal (ms, mt) lifted to the hemisphere. */
void oracle_shadow_masking(const double *Omega_all, int N, const double *q, const double *wi, const double *wo,
                           int64_t k0, int64_t k1, double *G)
{
    for (int64_t k = k0; k < k1; ++k) {
        double O[3];
        const double *qq = q + 7 * k;
        if (!ggx_omega_at(Omega_all, N, qq[0], qq[1], qq[2], qq[4], O)) {
            G[k] = NAN;
            continue;
        }
        const double *a = wi + 3 * k, *b = wo + 3 * k;
        double mz = sqrt(fmax(0.0, 1.0 - qq[5] * qq[5] - qq[6] * qq[6]));
        double ci = qq[5] * a[0] + qq[6] * a[1] + mz * a[2], co = qq[5] * b[0] + qq[6] * b[1] + mz * b[2];
        if (!(ci > 0.0 && co > 0.0)) {
            G[k] = 0.0;
            continue;
        }
        double li = ggx_P(O, a) / a[2] - 1.0, lo = ggx_P(O, b) / b[2] - 1.0;
        G[k] = 1.0 / (1.0 + li + lo);
    }
}
