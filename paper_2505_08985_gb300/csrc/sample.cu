// P-NDF sampling (Sec. 3, Eq. 6).
//
// A normal is drawn from D by drawing a uv point from the footprint kernel,
// u ~ k_r(u - x), and querying the map there, m = n(u) (Eq. 3); with the
// Jacobian clamp of Eq. 6 a fine triangle whose |cross| is below eps stands
// for its equilateral replacement (area eps / 2, centred at its normal
// centroid, vertex k at 90 + 120 k degrees, vertices in the uv order), so the
// density of the sampled normals is the clamped D over the kernel mass.
//
// u comes from the caller's two uniforms by the inverse CDF in the whitened
// frame v, u = x + L v with S = L L^T (Cholesky):
//   Gaussian cut at q = 16: |v|^2 = -2 ln(1 - U1 (1 - e^-8)), angle 2 pi U2;
//   disk (q <= 1.5^2): |v| = 1.5 sqrt(U1), angle 2 pi U2;
//   box (|v|_inf <= 1.5): v = 1.5 (2 U1 - 1, 2 U2 - 1).
// One thread per sample; the position arithmetic is FP64 (a handful of
// operations against four texel loads), so the triangle chosen for u agrees
// with an FP64 reference except at exact ties.
#include <math.h>

#include "common.cuh"

namespace pndf {
namespace {

template <int TFMT>
__device__ __forceinline__ float2 texel_s(const MapDesc &d, int i, int j)
{
    size_t idx = size_t(j) * d.n + i;
    if (TFMT == PNDF_TEXEL_F32X2) return __ldg(reinterpret_cast<const float2 *>(d.texels) + idx);
    return __half22float2(__ldg(reinterpret_cast<const __half2 *>(d.texels) + idx));
}

template <int TFMT>
__global__ void sample_kernel(MapDesc d, const pndf_query *__restrict__ q, const float *__restrict__ uni, int64_t n,
                              int kernel, float jac_eps, float *__restrict__ m_out, uint32_t *__restrict__ tri_out,
                              uint32_t *__restrict__ flags_out)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const pndf_query r = q[k];
        const double x = r.x, y = r.y, sxx = r.sxx, sxy = r.sxy, syy = r.syy;
        const double det = sxx * syy - sxy * sxy;
        float mx = 0.f, my = 0.f;
        uint32_t tri_id = 0xffffffffu, fl = 0;
        if (!(sxx > 0.0) || !(syy > 0.0) || !(det > 0.0) || !isfinite(det) || !isfinite(x) || !isfinite(y)) {
            fl = PNDF_SF_INVALID;
        } else {
            const double u1 = uni[2 * k], u2 = uni[2 * k + 1];
            double v1, v2;
            if (kernel == PNDF_KERNEL_BOX) {
                v1 = 1.5 * (2.0 * u1 - 1.0);
                v2 = 1.5 * (2.0 * u2 - 1.0);
            } else {
                const double rad = kernel == PNDF_KERNEL_DISK ? 1.5 * sqrt(u1)
                                                              : sqrt(-2.0 * log(1.0 - u1 * (1.0 - exp(-8.0))));
                double sn, cs;
                sincospi(2.0 * u2, &sn, &cs);
                v1 = rad * cs;
                v2 = rad * sn;
            }
            const double l11 = sqrt(sxx), l21 = sxy / l11, l22 = sqrt(syy - l21 * l21);
            const double ux = x + l11 * v1, uy = y + l21 * v1 + l22 * v2;
            const double fi = floor(ux), fj = floor(uy);
            if (!(fi >= 0.0 && fj >= 0.0 && fi <= d.n - 2 && fj <= d.n - 2)) {
                fl = PNDF_SF_OUTSIDE;
            } else {
                const int i = int(fi), j = int(fj);
                const double fu = ux - fi, fv = uy - fj;
                const int tri = fu + fv < 1.0 ? 0 : 1;
                // Tab. 1 order: (u0, u1, u2) or (u3, u2, u1), barycentric weights of u
                float2 na, nb, nc;
                double l0, lb, lc;
                if (tri == 0) {
                    na = texel_s<TFMT>(d, i, j);
                    nb = texel_s<TFMT>(d, i + 1, j);
                    nc = texel_s<TFMT>(d, i, j + 1);
                    l0 = 1.0 - fu - fv;
                    lb = fu;
                    lc = fv;
                } else {
                    na = texel_s<TFMT>(d, i + 1, j + 1);
                    nb = texel_s<TFMT>(d, i, j + 1);
                    nc = texel_s<TFMT>(d, i + 1, j);
                    l0 = fu + fv - 1.0;
                    lb = 1.0 - fu;
                    lc = 1.0 - fv;
                }
                double ax = na.x, ay = na.y, bx = nb.x, by = nb.y, cx = nc.x, cy = nc.y;
                const double cr = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
                if (jac_eps > 0.f && fabs(cr) < double(jac_eps)) {
                    const double gx = (ax + bx + cx) / 3.0, gy = (ay + by + cy) / 3.0;
                    const double rho = sqrt(2.0 * double(jac_eps) / sqrt(3.0)) / sqrt(3.0);
                    const double h = 0.5 * sqrt(3.0) * rho;
                    ax = gx;
                    ay = gy + rho;
                    bx = gx - h;
                    by = gy - 0.5 * rho;
                    cx = gx + h;
                    cy = gy - 0.5 * rho;
                }
                mx = float(l0 * ax + lb * bx + lc * cx);
                my = float(l0 * ay + lb * by + lc * cy);
                tri_id = 2u * (uint32_t(j) * uint32_t(d.n - 1) + uint32_t(i)) + uint32_t(tri);
            }
        }
        m_out[2 * k] = mx;
        m_out[2 * k + 1] = my;
        if (tri_out) tri_out[k] = tri_id;
        if (flags_out) flags_out[k] = fl;
    }
}

}  // namespace

cudaError_t launch_sample(const pndf_hierarchy *h, const pndf_query *q, const float *u, int64_t n, int kernel,
                          float jac_eps, float *m, uint32_t *tri, uint32_t *flags, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + 255) / 256;
    if (blocks > int64_t(sms) * 16) blocks = int64_t(sms) * 16;
    if (h->d.texel_fmt == PNDF_TEXEL_F32X2)
        sample_kernel<PNDF_TEXEL_F32X2><<<unsigned(blocks), 256, 0, s>>>(h->d, q, u, n, kernel, jac_eps, m, tri, flags);
    else
        sample_kernel<PNDF_TEXEL_F16X2><<<unsigned(blocks), 256, 0, s>>>(h->d, q, u, n, kernel, jac_eps, m, tri, flags);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pndf
