// Visible part of one normal triangle for the projected area (Eq. 10-11,
// Alg. 1, App. B), the general path: triangles that are only partly visible,
// thin slivers and triangles whose normals collapsed onto a segment.
//
// Notation.  m = (m_x, m_y) is a projected normal, z(m) = sqrt(1 - |m|^2) the
// height of m~ on the hemisphere, w = (w_x, w_y, w_z) the unit direction
// (w_z > 0).  In the frame rotated so w = (w_r, 0, w_z), a normal (x, y) sees
// w when w_r x + w_z z >= 0.  Every normal with x >= 0 does; for x < 0 the
// condition is (x / w_z)^2 + y^2 <= 1.  So in the scaled frame S(x, y) =
// (x / w_z, y) the boundary of the visible region is the left half of the
// unit circle, which is where Alg. 1 clips a triangle edge.
//
// The quantity integrated over the visible part of the normal triangle is
// g(m) = max(w . m~, 0) / z(m) = w_z + w_r x / z (Eq. 10), and with f = w_z x
// - w_r z (so that df/dx = g) Stokes' theorem turns the area integral into
// the counter-clockwise boundary integral of f dy (Eq. 11).  This file
// evaluates that boundary integral in a form that stays accurate when the
// visible part is small:
//
//   V = sum over the boundary's corner polygon of the trapezoid value of f dy
//       (written as a fan of 2 x 2 determinants of corner differences, so
//       nothing depends on absolute positions)
//     + for each straight piece p -> q: -w_r (y_q - y_p) H, H being how far
//       the mean of z along the chord exceeds (z_p + z_q) / 2 (App. B, the
//       line-segment integral of the square root, in angle form)
//     + for each piece of the unit circle between angles phi_s and phi_e:
//       (delta - sin delta) / 2 with delta = phi_e - phi_s (on that circle
//       f = cos phi and dy = cos phi dphi, so the arc exceeds its chord's
//       trapezoid by exactly this).
//
// The polygon's corners are kept as offsets from the first vertex, the clip
// parameters along each edge come from a line-circle intersection in the
// scaled frame (foot of the perpendicular and half chord), and the circle
// angles from atan2 of the corner pair.  All of it runs in FP64: the visible
// part of a clipped triangle can be many orders of magnitude smaller than
// the triangle, and an FP32 evaluation of the same sums (tried, with a
// rounding estimate) could not be trusted to 1e-5 there.
//
// Triangles whose normal-space area is (numerically) zero are the segment
// form of Eq. 13, integrated in closed form (collapsed_visible).
//
// Compiles as CUDA device code and as plain host C++ (for CPU checks of the
// arithmetic).
#pragma once

#ifdef __CUDACC__
#define PNDF_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define PNDF_HD inline
#endif

namespace pndf {
namespace vis {

PNDF_HD float vsqrt(float x) { return sqrtf(x); }
PNDF_HD double vsqrt(double x) { return sqrt(x); }
PNDF_HD float vatan2(float y, float x) { return atan2f(y, x); }
PNDF_HD double vatan2(double y, double x) { return atan2(y, x); }
PNDF_HD float vsin(float x) { return sinf(x); }
PNDF_HD double vsin(double x) { return sin(x); }
PNDF_HD float vfma(float a, float b, float c) { return fmaf(a, b, c); }
PNDF_HD double vfma(double a, double b, double c) { return fma(a, b, c); }
PNDF_HD float vabs(float x) { return fabsf(x); }
PNDF_HD double vabs(double x) { return fabs(x); }
template <typename R> PNDF_HD R vmax(R a, R b) { return a > b ? a : b; }
template <typename R> PNDF_HD R vmin(R a, R b) { return a < b ? a : b; }

// a * b - c * d with one FMA correction (Kahan).
template <typename R>
PNDF_HD R dprod(R a, R b, R c, R d)
{
    const R cd = c * d;
    return vfma(a, b, -cd) + vfma(-c, d, cd);
}

// t - sin t without cancellation: its Taylor series t^3/6 (1 - t^2/20 (1 -
// t^2/42 (...))) for |t| < 1 (six factors: relative truncation below 5e-11
// there, 2e-17 at |t| < 0.25), else directly.
template <typename R>
PNDF_HD R t_minus_sin(R t)
{
    if (vabs(t) < R(1)) {
        const R u = t * t;
        R s = R(1) - u * R(1.0 / 210.0);
        s = R(1) - u * R(1.0 / 156.0) * s;
        s = R(1) - u * R(1.0 / 110.0) * s;
        s = R(1) - u * R(1.0 / 72.0) * s;
        s = R(1) - u * R(1.0 / 42.0) * s;
        s = R(1) - u * R(1.0 / 20.0) * s;
        return t * u * R(1.0 / 6.0) * s;
    }
    return t - vsin(t);
}

// z(q) - z(p) for z(m) = sqrt(1 - |m|^2), from the difference of squares:
// (|p|^2 - |q|^2) / (z_p + z_q), with q - p given (dx, dy) and the sum q + p.
template <typename R>
PNDF_HD R zdelta(R dx, R dy, R sx, R sy, R zp, R zq)
{
    return -vfma(dx, sx, dy * sy) / (zp + zq);
}

// Excess of the mean of z over the chord p -> p + e above the chord's
// trapezoid value (z_p + z_q) / 2.  Along the line, with u the signed
// distance from the foot of the perpendicular and r^2 = 1 - (distance of the
// line from the origin)^2, z = sqrt(r^2 - u^2) = r cos psi with u = r sin psi,
// and the integral of z du is (r^2 / 2)(psi + sin psi cos psi).  Taking away
// the trapezoid leaves (r^2 / 2)(dpsi - sin dpsi) over the chord length, with
// dpsi the angle between (u_p, z_p) and (u_q, z_q): atan2 of their cross and
// dot products.  The cross product u_q z_p - u_p z_q is formed as
// L (r^2 + dot) / (z_p + z_q), which has no cancellation.
template <typename R>
PNDF_HD R chord_excess(R ex, R ey, R px, R py, R zp, R zq)
{
    const R L2 = vfma(ex, ex, ey * ey);
    if (!(L2 > R(0))) return R(0);
    const R L = vsqrt(L2);
    const R up = vfma(ex, px, ey * py) / L;
    const R uq = up + L;
    const R r2 = vfma(zp, zp, up * up);
    const R dot = vfma(zp, zq, up * uq);
    const R crs = L * (r2 + dot) / (zp + zq);
    return R(0.5) * r2 * t_minus_sin(vatan2(crs, dot)) / L;
}

// Direction with its rotation to w_y = 0 and the scaled frame, in FP64.
struct DirD {
    double wx, wy, wz;  // unit direction, w_z > 0
    double cs, sn, wr;  // (w_x, w_y) = w_r (cs, sn); cs = 1, sn = 0 when w_r = 0
    double iwz;         // 1 / w_z
};

// From a direction given to single precision: normalised, since the clip
// circle and the arc terms hold for a unit vector only.
PNDF_HD DirD make_dir(double wx, double wy, double wz)
{
    DirD d;
    const double n = sqrt(wx * wx + wy * wy + wz * wz);
    d.wx = wx / n;
    d.wy = wy / n;
    d.wz = wz / n;
    wx = d.wx;
    wy = d.wy;
    d.wr = sqrt(wx * wx + wy * wy);
    d.cs = d.wr > 0.0 ? wx / d.wr : 1.0;
    d.sn = d.wr > 0.0 ? wy / d.wr : 0.0;
    d.iwz = 1.0 / d.wz;
    return d;
}

// Scaled-frame position S(m) = (x / w_z, y) of a normal m (rotated frame).
PNDF_HD void scaled(const DirD &w, double mx, double my, double &X, double &Y)
{
    X = (w.cs * mx + w.sn * my) * w.iwz;
    Y = w.cs * my - w.sn * mx;
}

// Visibility of a normal from its scaled position: x >= 0, or inside the
// unit circle.
PNDF_HD bool sees(double X, double Y) { return X >= 0.0 || X * X + Y * Y <= 1.0; }

// Visible part [t0, t1] of the edge P + t D, t in [0, 1], between scaled
// points P and P + D with visibilities vp, vq (Alg. 1's clip, posed as a
// line-circle intersection).  Returns false when nothing of the edge is
// visible.  in / out: whether t0 / t1 were moved onto the circle.
//
// The line meets the unit circle where |P + t D| = 1: around the foot of the
// perpendicular t_f = -(P . D) / |D|^2 at half-width sqrt(|D|^2 - (P x
// D)^2) / |D|^2 (P x D / |D| is the line's distance from the origin).  The
// visible part of the line is the chord inside the circle joined to the
// half plane x >= 0 (a convex set); an edge that leaves the region leaves it
// at the far end of the chord, one that enters it enters at the near end,
// and an edge with both ends outside sees exactly the chord if the chord
// lies within the edge.
PNDF_HD bool edge_interval(double PX, double PY, double DX, double DY, bool vp, bool vq, double &t0, double &t1,
                           bool &in, bool &out)
{
    in = out = false;
    t0 = 0.0;
    t1 = 1.0;
    if (vp && vq) return true;
    const double dd = DX * DX + DY * DY;
    if (!(dd > 0.0)) return vp;  // a point edge: visible with its end point
    const double along = PX * DX + PY * DY;
    const double across = PX * DY - PY * DX;
    const double h2 = dd - across * across;
    const double half = h2 > 0.0 ? sqrt(h2) : 0.0;
    const double tn = (-along - half) / dd, tf = (-along + half) / dd;
    if (vp) {  // leaves the visible region at the far end of the chord
        t1 = tf < 0.0 ? 0.0 : (tf > 1.0 ? 1.0 : tf);
        out = true;
        return true;
    }
    if (vq) {  // enters it at the near end
        t0 = tn < 0.0 ? 0.0 : (tn > 1.0 ? 1.0 : tn);
        in = true;
        return true;
    }
    if (!(h2 > 0.0) || tn < 0.0 || tf > 1.0) return false;
    t0 = tn;
    t1 = tf;
    in = out = true;
    return true;
}

// A corner of the clipped boundary: its offset from the triangle's first
// vertex and its z.
template <typename R>
struct Corner {
    R ox, oy;  // offset from vertex a (unrotated)
    R z;       // z at the corner
};

// V_T / |cross(T)| for the normal triangle (a, b, c) and direction w, where
// V_T is the integral of g over the visible part of the triangle (Eq. 10)
// and cross(T) = (b - a) x (c - a): the mean of g over the uv triangle times
// its area 1/2.  Not for |cross| = 0 (collapsed_visible).  R = double on the
// device; the template lets host checks run the same steps in other
// precisions.
template <typename R>
PNDF_HD R tri_visible(float ax, float ay, float bx, float by, float cx, float cy, const DirD &w)
{
    // counter-clockwise order a, b, c
    R e1x = R(bx) - R(ax), e1y = R(by) - R(ay), e2x = R(cx) - R(ax), e2y = R(cy) - R(ay);
    R cr = dprod(e1x, e2y, e1y, e2x);
    if (cr < R(0)) {
        const float tx = bx, ty = by;
        bx = cx;
        by = cy;
        cx = tx;
        cy = ty;
        R t;
        t = e1x; e1x = e2x; e2x = t;
        t = e1y; e1y = e2y; e2y = t;
        cr = -cr;
    }
    const float vx[3] = {ax, bx, cx}, vy[3] = {ay, by, cy};
    // edges as vectors: b - a, c - b, a - c
    const R ex[3] = {e1x, R(cx) - R(bx), -e2x}, ey[3] = {e1y, R(cy) - R(by), -e2y};
    const R ox[3] = {R(0), e1x, e2x}, oy[3] = {R(0), e1y, e2y};

    // clip each edge in FP64
    double X[3], Y[3];
    bool vis[3];
    for (int k = 0; k < 3; ++k) {
        scaled(w, double(vx[k]), double(vy[k]), X[k], Y[k]);
        vis[k] = sees(X[k], Y[k]);
    }
    bool alive[3], cl_in[3], cl_out[3];
    R t0[3], t1[3];
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1;
        double dX, dY;
        scaled(w, double(vx[k1]) - double(vx[k]), double(vy[k1]) - double(vy[k]), dX, dY);
        double a0, a1;
        alive[k] = edge_interval(X[k], Y[k], dX, dY, vis[k], vis[k1], a0, a1, cl_in[k], cl_out[k]);
        t0[k] = R(a0);
        t1[k] = R(a1);
    }

    // corners: the start of each visible piece, and its end where clipped
    const R wz = R(w.wz), wr = R(w.wr), cs = R(w.cs), sn = R(w.sn);
    const R axr = R(ax), ayr = R(ay);
    Corner<R> cor[6];
    int nc = 0;
    R curv = R(0);
    for (int k = 0; k < 3; ++k)
        if (alive[k]) {
            // piece from p = v_k + t0 e_k to q = v_k + t1 e_k
            const R px = vfma(t0[k], ex[k], ox[k]), py = vfma(t0[k], ey[k], oy[k]);
            const R qx = vfma(t1[k], ex[k], ox[k]), qy = vfma(t1[k], ey[k], oy[k]);
            const R zp = vsqrt(vmax(R(0), R(1) - vfma(axr + px, axr + px, (ayr + py) * (ayr + py))));
            const R zq = vsqrt(vmax(R(0), R(1) - vfma(axr + qx, axr + qx, (ayr + qy) * (ayr + qy))));
            cor[nc++] = Corner<R>{px, py, zp};
            if (cl_out[k]) cor[nc++] = Corner<R>{qx, qy, zq};
            // the chord's excess over its trapezoid, along the straight piece
            const R dxp = qx - px, dyp = qy - py;
            const R dyr = cs * dyp - sn * dxp;
            curv -= wr * dyr * chord_excess(dxp, dyp, axr + px, ayr + py, zp, zq);
        }
    if (nc == 0) return R(0);
    // circle pieces: from each clipped end to the start of the next visible piece
    for (int k = 0; k < 3; ++k) {
        if (!alive[k] || !cl_out[k]) continue;
        int nx = k;
        for (int s = 1; s <= 3; ++s) {
            const int j = (k + s) % 3;
            if (alive[j]) {
                nx = j;
                break;
            }
        }
        // scaled positions of the exit point and the next entry point
        const double sxk = double(vx[k]) + double(t1[k]) * (double(vx[(k + 1) % 3]) - double(vx[k]));
        const double syk = double(vy[k]) + double(t1[k]) * (double(vy[(k + 1) % 3]) - double(vy[k]));
        const double exk = double(vx[nx]) + double(t0[nx]) * (double(vx[(nx + 1) % 3]) - double(vx[nx]));
        const double eyk = double(vy[nx]) + double(t0[nx]) * (double(vy[(nx + 1) % 3]) - double(vy[nx]));
        double SX, SY, EX, EY;
        scaled(w, sxk, syk, SX, SY);
        scaled(w, exk, eyk, EX, EY);
        curv += R(0.5) * t_minus_sin(vatan2(R(SX * EY - SY * EX), R(SX * EX + SY * EY)));
    }
    // fan of the corner polygon from corner 0: the trapezoid sums of f dy
    R fan = R(0);
    const R o0x = cor[0].ox, o0y = cor[0].oy, z0 = cor[0].z;
    R pf = R(0), py_ = R(0);
    for (int i = 1; i < nc; ++i) {
        const R dx = cor[i].ox - o0x, dy = cor[i].oy - o0y;
        const R sx = R(2) * axr + cor[i].ox + o0x, sy = R(2) * ayr + cor[i].oy + o0y;
        const R dz = zdelta(dx, dy, sx, sy, z0, cor[i].z);
        const R xr = vfma(cs, dx, sn * dy), yr = vfma(cs, dy, -sn * dx);
        const R df = vfma(wz, xr, -wr * dz);
        if (i >= 2) fan += R(0.5) * dprod(pf, yr, df, py_);
        pf = df;
        py_ = yr;
    }
    return (fan + curv) / cr;
}

// The segment form of Eq. 13 for a triangle whose normals (a, b, c) lie on
// one line (|cross| numerically zero): the mean over the uv triangle (area
// 1/2) of g(n(u)), times 1/2.  With P, Q the farthest pair of normals and M
// the third, n(u) runs along P -> Q at parameter t(u), which is affine on the
// uv triangle with values 0, 1 and t_M at the corners; a uniform point of the
// triangle therefore has the triangular density 2 t / t_M on [0, t_M] and 2 (1
// - t) / (1 - t_M) on [t_M, 1], and the result is the integral of
// lambda(t) g over the visible part of the segment, lambda = t / t_M or (1 -
// t) / (1 - t_M).  Along the line, at arc length s from the foot of the
// perpendicular F (r^2 = 1 - |F|^2), g = w_z + (alpha + beta s) / sqrt(r^2 -
// s^2) with alpha = w_xy . F, beta = w_xy . d; lambda is linear in s, so each
// piece is an integral of a quadratic in s over sqrt(r^2 - s^2), in closed
// form with s = r sin psi: 1 -> psi, s -> -sqrt(r^2 - s^2), s^2 -> (r^2 / 2)
// (psi - sin psi cos psi).  All in FP64.
PNDF_HD double collapsed_visible(float ax, float ay, float bx, float by, float cx, float cy, const DirD &w)
{
    const double px0[3] = {ax, bx, cx}, py0[3] = {ay, by, cy};
    int ip = 0, iq = 1, im = 2;
    double best = -1.0;
    for (int i = 0; i < 3; ++i) {
        const int j = i == 2 ? 0 : i + 1;
        const double d2 = (px0[j] - px0[i]) * (px0[j] - px0[i]) + (py0[j] - py0[i]) * (py0[j] - py0[i]);
        if (d2 > best) {
            best = d2;
            ip = i;
            iq = j;
            im = 3 - i - j;
        }
    }
    const double Px = px0[ip], Py = py0[ip];
    if (best == 0.0) {  // one normal: g there, over the uv area 1/2
        const double z = sqrt(fmax(0.0, 1.0 - Px * Px - Py * Py));
        const double g = w.wz + (w.wx * Px + w.wy * Py) / z;
        return g > 0.0 ? 0.5 * g : 0.0;
    }
    const double Dx = px0[iq] - Px, Dy = py0[iq] - Py;
    const double len = sqrt(best);
    double tM = ((px0[im] - Px) * Dx + (py0[im] - Py) * Dy) / best;
    tM = tM < 0.0 ? 0.0 : (tM > 1.0 ? 1.0 : tM);
    // visible interval of P -> Q
    double SPX, SPY, SDX, SDY, SQX, SQY;
    scaled(w, Px, Py, SPX, SPY);
    scaled(w, px0[iq], py0[iq], SQX, SQY);
    scaled(w, Dx, Dy, SDX, SDY);
    double v0, v1;
    bool ci, co;
    if (!edge_interval(SPX, SPY, SDX, SDY, sees(SPX, SPY), sees(SQX, SQY), v0, v1, ci, co)) return 0.0;
    // arc-length frame along the line: unit direction d, foot F, r^2
    const double dx = Dx / len, dy = Dy / len;
    const double sP = Px * dx + Py * dy;
    const double Fx = Px - sP * dx, Fy = Py - sP * dy;
    const double r2 = 1.0 - (Fx * Fx + Fy * Fy);
    const double alpha = w.wx * Fx + w.wy * Fy, beta = w.wx * dx + w.wy * dy;
    double sum = 0.0;
    for (int piece = 0; piece < 2; ++piece) {
        const double lo = fmax(v0, piece == 0 ? 0.0 : tM), hi = fmin(v1, piece == 0 ? tM : 1.0);
        if (!(hi > lo)) continue;
        // lambda(t) = l0 + l1 t on this piece
        const double l0 = piece == 0 ? 0.0 : 1.0 / (1.0 - tM);
        const double l1 = piece == 0 ? 1.0 / tM : -1.0 / (1.0 - tM);
        // the w_z part: w_z times the integral of lambda
        sum += w.wz * (hi - lo) * (l0 + 0.5 * l1 * (lo + hi));
        // in s = sP + t len: lambda = m0 + m1 s
        const double m1 = l1 / len, m0 = l0 - m1 * sP;
        const double c0 = m0 * alpha, c1 = m0 * beta + m1 * alpha, c2 = m1 * beta;
        const double sa = sP + lo * len, sb = sP + hi * len;
        const double za = sqrt(fmax(0.0, r2 - sa * sa)), zb = sqrt(fmax(0.0, r2 - sb * sb));
        const double dpsi = atan2(sb * za - sa * zb, za * zb + sa * sb);
        const double dz = (sa - sb) * (sa + sb) / (za + zb);  // zb - za
        const double J0 = dpsi, J1 = -dz, J2 = 0.5 * r2 * dpsi - 0.5 * (sb * zb - sa * za);
        // dt = ds / len
        sum += (c0 * J0 + c1 * J1 + c2 * J2) / len;
    }
    return sum;
}

}  // namespace vis
}  // namespace pndf
