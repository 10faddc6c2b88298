// GGX projected-area fit per mip node (Eq. 12) and shadow-masking (Sec. 4.3):
// the device object and its launchers (projarea.cu).
#pragma once

#include "common.cuh"

namespace pndf {
constexpr int kGgxDirs = 16;  // fit directions: azimuths 2 pi k / 16 at w_z = 0.3
constexpr float kGgxWz = 0.3f;
}  // namespace pndf

// Fitted Omega = (O_xx, O_xy, O_yy, unused) per node of levels 2..L in the
// boxes' Morton order; NaN where the node has a quad outside the map.
struct pndf_ggx {
    int device;
    int n, L;
    float4 *omega[pndf::kMaxLevels];
    void *mem;
    size_t bytes;
};

namespace pndf {
// Fit every node of h into g (g->omega allocated by the caller).
pndf_status launch_ggx_build(const pndf_hierarchy *h, pndf_ggx *g, cudaStream_t s);
// Lambda'(w) per request, or the height-correlated G when wo != nullptr.
cudaError_t launch_ggx_eval(const pndf_ggx *g, const pndf_query *q, const float *wi, const float *wo, int64_t n,
                            float *out, cudaStream_t s);
// Level l of the fit in row-major node order (3 floats per node).
cudaError_t launch_ggx_copy(const pndf_ggx *g, int l, float *out, cudaStream_t s);
}  // namespace pndf
